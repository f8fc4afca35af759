"""ctypes binding of libnhmf.so: the C entry points under the same names, plus `Problem`.

Arguments are marshalled only: tensors become device pointers (`data_ptr()`), the stream is
torch's current CUDA stream.  Every computation runs in the library's CUDA kernels; if the
library is missing the import of a function raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnhmf.so")

NHMF_OK = 0
(NHMF_ERR_ARG, NHMF_ERR_CUDA, NHMF_ERR_OOM, NHMF_ERR_NONPOS_J, NHMF_ERR_NONFINITE, NHMF_ERR_BREAKDOWN,
 NHMF_ERR_NOT_CONVERGED, NHMF_ERR_STATE) = range(1, 9)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NONPOS_J",
                5: "ERR_NONFINITE", 6: "ERR_BREAKDOWN", 7: "ERR_NOT_CONVERGED", 8: "ERR_STATE"}
NHMF_FP64, NHMF_FP32, NHMF_DF64 = 0, 1, 2
NHMF_ON_THE_FLY, NHMF_CACHED, NHMF_SPATIAL = 0, 1, 2
NHMF_BC_NONE, NHMF_BC_CLAMP_X0, NHMF_BC_COMPRESSION = 0, 1, 2
NHMF_CACHE_FP64, NHMF_CACHE_FP32, NHMF_CACHE_DF64, NHMF_CACHE_SPATIAL = 1, 2, 4, 8
NHMF_KIND_APPLY, NHMF_KIND_CACHE, NHMF_KIND_RESIDUAL, NHMF_KIND_DIAGONAL = 0, 1, 2, 3
NHMF_INJECT_NAN_DU, NHMF_INJECT_CG_STALL, NHMF_INJECT_UNET_GARBAGE, NHMF_INJECT_UNKNOWN = 1, 2, 4, 1 << 30


class NhmfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class nhmf_params(ctypes.Structure):
    _fields_ = [("n_el", ctypes.c_int), ("degree", ctypes.c_int), ("mu", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("bc", ctypes.c_int), ("top_uz", ctypes.c_double),
                ("model", ctypes.c_int)]


NHMF_SOLVER_JACOBI_CG, NHMF_SOLVER_MIXED_FCG, NHMF_SOLVER_LEARNED_FCG, NHMF_SOLVER_MIXED_LEARNED = 0, 1, 2, 3
NHMF_SOLVER_GMG, NHMF_SOLVER_MIXED_GMG, NHMF_SOLVER_MIXED_GMG_LEARNED = 4, 5, 6
NHMF_MAX_STEPS = 64


class nhmf_solve_opts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("strategy", ctypes.c_int), ("load_steps", ctypes.c_int),
                ("first_step", ctypes.c_int), ("last_step", ctypes.c_int), ("compression", ctypes.c_double),
                ("newton_rtol", ctypes.c_double), ("newton_max_iter", ctypes.c_int),
                ("max_backtracks", ctypes.c_int), ("linear_rtol", ctypes.c_double),
                ("linear_max_iter", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("inner_max_iter", ctypes.c_int), ("check_every", ctypes.c_int),
                ("record_pairs", ctypes.c_int), ("cg_pair_every", ctypes.c_int),
                ("learned_stall_window", ctypes.c_int), ("learned_stall_factor", ctypes.c_double),
                ("synthetic_pairs", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("smoother_degree", ctypes.c_int), ("smoother_range", ctypes.c_double),
                ("outer_apply", ctypes.c_int)]


class nhmf_solve_stats(ctypes.Structure):
    _fields_ = [("steps_done", ctypes.c_int), ("newton_iters", ctypes.c_int * NHMF_MAX_STEPS),
                ("linear_iters", ctypes.c_longlong * NHMF_MAX_STEPS),
                ("inner_iters", ctypes.c_longlong * NHMF_MAX_STEPS),
                ("fallbacks", ctypes.c_int * NHMF_MAX_STEPS),
                ("rel_residual", ctypes.c_double * NHMF_MAX_STEPS),
                ("seconds", ctypes.c_double * NHMF_MAX_STEPS),
                ("total_linear_iters", ctypes.c_longlong), ("total_inner_iters", ctypes.c_longlong),
                ("total_seconds", ctypes.c_double)]

    def as_dict(self):
        k = self.steps_done
        return {"steps_done": k, "newton_iters": list(self.newton_iters[:k]),
                "linear_iters": list(self.linear_iters[:k]), "inner_iters": list(self.inner_iters[:k]),
                "fallbacks": list(self.fallbacks[:k]), "rel_residual": list(self.rel_residual[:k]),
                "seconds": list(self.seconds[:k]), "total_linear_iters": self.total_linear_iters,
                "total_inner_iters": self.total_inner_iters, "total_seconds": self.total_seconds}


_lib = None
_P = ctypes.c_void_p
_SIGS = {
    "nhmf_create": (ctypes.c_int, [ctypes.POINTER(nhmf_params), ctypes.POINTER(_P)]),
    "nhmf_destroy": (None, [_P]),
    "nhmf_num_dofs": (ctypes.c_size_t, [_P]),
    "nhmf_last_error": (ctypes.c_char_p, [_P]),
    "nhmf_set_linearization": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "nhmf_tangent_apply": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "nhmf_tangent_apply_at": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "nhmf_residual": (ctypes.c_int, [_P, _P, _P, _P]),
    "nhmf_diagonal": (ctypes.c_int, [_P, _P, _P]),
    "nhmf_check_status": (ctypes.c_int, [_P, _P]),
    "nhmf_set_material_factors": (ctypes.c_int, [_P, _P, _P]),
    "nhmf_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "nhmf_solve_opts_default": (None, [ctypes.POINTER(nhmf_solve_opts)]),
    "nhmf_solve": (ctypes.c_int, [_P, ctypes.POINTER(nhmf_solve_opts), _P, ctypes.POINTER(nhmf_solve_stats), _P]),
    "nhmf_unet_create": (ctypes.c_int, [_P, ctypes.c_int]),
    "nhmf_unet_num_params": (ctypes.c_size_t, [_P]),
    "nhmf_unet_num_pairs": (ctypes.c_int, [_P]),
    "nhmf_unet_set_params": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "nhmf_unet_get_params": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "nhmf_unet_forward": (ctypes.c_int, [_P, _P, _P, _P]),
    "nhmf_unet_loss_grad": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double), _P, _P]),
    "nhmf_unet_precondition": (ctypes.c_int, [_P, _P, _P, _P]),
    "nhmf_unet_record_pair": (ctypes.c_int, [_P, _P, _P, _P]),
    "nhmf_unet_train": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), _P]),
    "nhmf_linear_solve_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_int, _P, _P,
                                                 ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double), _P]),
    "nhmf_linear_solve": (ctypes.c_int, [_P, ctypes.POINTER(nhmf_solve_opts), _P, _P,
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_double), _P]),
    "nhmf_profile_read": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_longlong)]),
    "nhmf_measure_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "nhmf_set_inject": (ctypes.c_int, [_P, ctypes.c_uint]),
    "nhmf_inject_pending": (ctypes.c_uint, [_P]),
    "nhmf_parse_inject": (ctypes.c_uint, [ctypes.c_char_p]),
    "nhmf_set_metrics_log": (ctypes.c_int, [_P, ctypes.c_char_p]),
}


def lib():
    """The loaded library; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(ctx, st):
    if st != NHMF_OK:
        raise NhmfError(st, lib().nhmf_last_error(ctx).decode())


# ---- the C entry points, same names ---------------------------------------------------
NHMF_MODEL_COMPRESSIBLE, NHMF_MODEL_SPLIT = 0, 1


def nhmf_create(n_el, degree, mu, lam, bc, top_uz=0.0, model=0):
    prm = nhmf_params(n_el, degree, mu, lam, bc, top_uz, model)
    ctx = _P()
    st = lib().nhmf_create(ctypes.byref(prm), ctypes.byref(ctx))
    if st != NHMF_OK:
        raise NhmfError(st, "nhmf_create failed")
    return ctx


def nhmf_destroy(ctx):
    lib().nhmf_destroy(ctx)


def nhmf_num_dofs(ctx):
    return lib().nhmf_num_dofs(ctx)


def nhmf_last_error(ctx):
    return lib().nhmf_last_error(ctx).decode()


def nhmf_set_linearization(ctx, u, cache_mask=0, stream=None):
    _check(ctx, lib().nhmf_set_linearization(ctx, _ptr(u), cache_mask, _stream(stream)))


def nhmf_tangent_apply(ctx, precision, strategy, du, v, stream=None):
    _check(ctx, lib().nhmf_tangent_apply(ctx, precision, strategy, _ptr(du), _ptr(v), _stream(stream)))


def nhmf_tangent_apply_at(ctx, u, du, v, stream=None):
    _check(ctx, lib().nhmf_tangent_apply_at(ctx, _ptr(u), _ptr(du), _ptr(v), _stream(stream)))


def nhmf_residual(ctx, u, r, stream=None):
    _check(ctx, lib().nhmf_residual(ctx, _ptr(u), _ptr(r), _stream(stream)))


def nhmf_diagonal(ctx, d, stream=None):
    _check(ctx, lib().nhmf_diagonal(ctx, _ptr(d), _stream(stream)))


def nhmf_set_material_factors(ctx, factors, stream=None):
    """factors: CUDA FP64 tensor of N^3 per-element factors (natural order), or None."""
    _check(ctx, lib().nhmf_set_material_factors(ctx, _ptr(factors) if factors is not None else None,
                                                _stream(stream)))


def nhmf_check_status(ctx, stream=None):
    _check(ctx, lib().nhmf_check_status(ctx, _stream(stream)))


def nhmf_profile_enable(ctx, enable):
    _check(ctx, lib().nhmf_profile_enable(ctx, int(bool(enable))))


def nhmf_profile_read(ctx, kind):
    """(elapsed_ms, launches) of the element kernels of one operator kind since the last read."""
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(ctx, lib().nhmf_profile_read(ctx, kind, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def nhmf_set_inject(ctx, flags):
    _check(ctx, lib().nhmf_set_inject(ctx, flags))


def nhmf_inject_pending(ctx):
    return lib().nhmf_inject_pending(ctx)


def nhmf_parse_inject(spec):
    return lib().nhmf_parse_inject(spec.encode() if spec is not None else None)


def nhmf_set_metrics_log(ctx, path):
    _check(ctx, lib().nhmf_set_metrics_log(ctx, path.encode() if path else None))


def nhmf_measure_fma_peak(precision):
    """Measured FMA throughput of the current device in TFLOP/s (NHMF_FP64 or NHMF_FP32)."""
    out = ctypes.c_double()
    st = lib().nhmf_measure_fma_peak(precision, ctypes.byref(out))
    if st != NHMF_OK:
        raise NhmfError(st, "measure_fma_peak")
    return out.value


def nhmf_solve_opts_default(**overrides):
    o = nhmf_solve_opts()
    lib().nhmf_solve_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def nhmf_solve(ctx, opts, u, stream=None):
    """Run the Newton load steps; returns the stats (raises NhmfError on failure, with the
    partial stats attached as `.stats`)."""
    stats = nhmf_solve_stats()
    st = lib().nhmf_solve(ctx, ctypes.byref(opts), _ptr(u), ctypes.byref(stats), _stream(stream))
    if st != NHMF_OK:
        err = NhmfError(st, lib().nhmf_last_error(ctx).decode())
        err.stats = stats.as_dict()
        raise err
    return stats.as_dict()


def nhmf_linear_solve(ctx, opts, b, x, stream=None):
    """(outer iterations, inner iterations, true relative residual)."""
    it, inner, rel = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
    _check(ctx, lib().nhmf_linear_solve(ctx, ctypes.byref(opts), _ptr(b), _ptr(x), ctypes.byref(it),
                                        ctypes.byref(inner), ctypes.byref(rel), _stream(stream)))
    return it.value, inner.value, rel.value


def nhmf_linear_solve_noalloc(ctx, strategy, rtol, max_iter, b, x, stream=None):
    """Jacobi-CG solve with static scratch (no allocation); (iterations, true relative residual)."""
    it, rel = ctypes.c_longlong(), ctypes.c_double()
    _check(ctx, lib().nhmf_linear_solve_noalloc(ctx, strategy, rtol, max_iter, _ptr(b), _ptr(x), ctypes.byref(it),
                                                ctypes.byref(rel), _stream(stream)))
    return it.value, rel.value


def _host_f32(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def nhmf_unet_create(ctx, pair_capacity=0):
    _check(ctx, lib().nhmf_unet_create(ctx, int(pair_capacity)))


def nhmf_unet_num_params(ctx):
    return lib().nhmf_unet_num_params(ctx)


def nhmf_unet_num_pairs(ctx):
    return lib().nhmf_unet_num_pairs(ctx)


def nhmf_unet_set_params(ctx, params):
    """params: host array-like of num_params floats (flat layout, see include/nhmf.h)."""
    a, p = _host_f32(params)
    _check(ctx, lib().nhmf_unet_set_params(ctx, p, a.size))


def nhmf_unet_get_params(ctx):
    import numpy as np
    out = np.empty(nhmf_unet_num_params(ctx), dtype=np.float32)
    _check(ctx, lib().nhmf_unet_get_params(ctx, out.ctypes.data_as(ctypes.c_void_p), out.size))
    return out


def nhmf_unet_forward(ctx, x, y, stream=None):
    _check(ctx, lib().nhmf_unet_forward(ctx, _ptr(x), _ptr(y), _stream(stream)))


def nhmf_unet_loss_grad(ctx, x, e, stream=None):
    """(loss, host FP32 gradient array)."""
    import numpy as np
    g = np.empty(nhmf_unet_num_params(ctx), dtype=np.float32)
    loss = ctypes.c_double()
    _check(ctx, lib().nhmf_unet_loss_grad(ctx, _ptr(x), _ptr(e), ctypes.byref(loss),
                                          g.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return loss.value, g


def nhmf_unet_precondition(ctx, r, z, stream=None):
    _check(ctx, lib().nhmf_unet_precondition(ctx, _ptr(r), _ptr(z), _stream(stream)))


def nhmf_unet_record_pair(ctx, r, e, stream=None):
    _check(ctx, lib().nhmf_unet_record_pair(ctx, _ptr(r), _ptr(e), _stream(stream)))


def nhmf_unet_train(ctx, epochs, lr, stream=None):
    """(mean loss of the first epoch, mean loss of the last epoch)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().nhmf_unet_train(ctx, int(epochs), float(lr), ctypes.byref(a), ctypes.byref(b), _stream(stream)))
    return a.value, b.value


class Problem:
    """One mesh + material on the current CUDA device (owns an nhmf context)."""

    def __init__(self, n_el, degree, mu, lam, bc, top_uz=0.0, model=0):
        self.n_el, self.degree, self.mu, self.lam, self.bc, self.model = n_el, degree, mu, lam, bc, model
        self.ctx = nhmf_create(n_el, degree, mu, lam, bc, top_uz, model)
        self.n_dofs = nhmf_num_dofs(self.ctx)

    @classmethod
    def from_workload(cls, w):
        return cls(w.n_el, w.degree, w.mu, w.lam, w.bc)

    def close(self):
        if self.ctx is not None:
            nhmf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_linearization(self, u, cache_mask=0):
        nhmf_set_linearization(self.ctx, u, cache_mask)

    def apply(self, du, v, precision=NHMF_FP64, strategy=NHMF_ON_THE_FLY):
        nhmf_tangent_apply(self.ctx, precision, strategy, du, v)
        return v

    def apply_at(self, u, du, v):
        """v = A(u) du on the fly in FP64 at the given u (no stored linearisation needed)."""
        nhmf_tangent_apply_at(self.ctx, u, du, v)
        return v

    def residual(self, u, r):
        nhmf_residual(self.ctx, u, r)
        return r

    def diagonal(self, d):
        nhmf_diagonal(self.ctx, d)
        return d

    def solve(self, u, **opts):
        return nhmf_solve(self.ctx, nhmf_solve_opts_default(**opts), u)

    def linear_solve(self, b, x, **opts):
        return nhmf_linear_solve(self.ctx, nhmf_solve_opts_default(**opts), b, x)
