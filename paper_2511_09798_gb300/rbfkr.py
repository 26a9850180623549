"""Thin ctypes binding of ``include/rbfkr.h`` (argument marshalling only).

Device buffers are passed as torch CUDA tensors (their ``data_ptr()``); every
step of the computation runs in ``librbfkr.so``.  Each function raises
``RbfError`` with the library's message when the C call fails.  There is no
fallback: if the shared library is missing or cannot be loaded, importing
functions from here raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librbfkr.so")

RBF_OK, RBF_ERR_INVALID, RBF_ERR_OOM, RBF_ERR_CUDA, RBF_ERR_TIMEOUT, RBF_ERR_UNSUPPORTED, RBF_ERR_INTERNAL = range(7)
RBF_FP64, RBF_MIXED = 0, 1
RBF_ASSEMBLED, RBF_MATRIX_FREE = 0, 1
RBF_GCV, RBF_LCURVE, RBF_FIXED, RBF_FIXED_T = 0, 1, 2, 3
RBF_FORM_C, RBF_FORM_EPS = 0, 1

STATUS_NAMES = {0: "RBF_OK", 1: "RBF_ERR_INVALID", 2: "RBF_ERR_OOM", 3: "RBF_ERR_CUDA",
                4: "RBF_ERR_TIMEOUT", 5: "RBF_ERR_UNSUPPORTED", 6: "RBF_ERR_INTERNAL"}


class RbfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("grid_j", C.c_int), ("grid_t_lo", C.c_double), ("grid_t_hi", C.c_double),
                ("breakdown_factor", C.c_double), ("cluster_tol", C.c_double),
                ("workspace_cap", C.c_int64), ("timing", C.c_int), ("svd_method", C.c_int),
                ("wait_budget", C.c_int64), ("fma_products", C.c_int)]


class Operator(C.Structure):
    _fields_ = [("d_nodes", C.c_void_p), ("n", C.c_int64), ("n_interior", C.c_int64),
                ("c", C.c_double), ("k", C.c_double), ("storage", C.c_int),
                ("precision", C.c_int), ("form", C.c_int), ("d_A", C.c_void_p), ("lda", C.c_int64)]


class GkbState(C.Structure):
    _fields_ = [("d_W", C.c_void_p), ("ldw", C.c_int64), ("d_Z", C.c_void_p), ("ldz", C.c_int64),
                ("d_alpha", C.c_void_p), ("d_beta", C.c_void_p), ("capacity", C.c_int),
                ("n", C.c_int64), ("steps_done", C.c_int), ("breakdown", C.c_int),
                ("c_hat", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("index", C.c_int), ("rank", C.c_int), ("steps", C.c_int),
                ("sigma1", C.c_double), ("eta", C.c_double), ("rho", C.c_double)]


class LearnedInfo(C.Structure):
    _fields_ = [("l_pred", C.c_int), ("t_pred", C.c_double), ("accepted", C.c_int), ("in_distribution", C.c_int),
                ("eta_change", C.c_double), ("steps", C.c_int), ("solve", SolveInfo)]


class Counters(C.Structure):
    _fields_ = [("launches", C.c_int64), ("product_launches", C.c_int64 * 2),
                ("product_ms", C.c_double * 2), ("product_busy_ms", C.c_double),
                ("reorth_launches", C.c_int64), ("reorth_ms", C.c_double)]


class Batch(C.Structure):
    _fields_ = [("count", C.c_int), ("n", C.POINTER(C.c_int64)), ("n_interior", C.POINTER(C.c_int64)),
                ("c", C.POINTER(C.c_double)), ("k", C.POINTER(C.c_double)), ("d_nodes", C.c_void_p),
                ("d_f", C.c_void_p), ("capacity", C.c_int), ("d_W", C.c_void_p), ("d_Z", C.c_void_p),
                ("d_alpha", C.c_void_p), ("d_beta", C.c_void_p), ("steps_done", C.POINTER(C.c_int)),
                ("breakdown", C.POINTER(C.c_int)), ("steps_limit", C.POINTER(C.c_int))]


class Tuning(C.Structure):
    _fields_ = [("mf_outputs_per_thread", C.c_int), ("mf_threads", C.c_int), ("candidates", C.c_int),
                ("best_ms", C.c_double), ("graph_kernels", C.c_int)]


class StopNet(C.Structure):
    _fields_ = [("d_params", C.c_void_p), ("d_feat_mean", C.c_void_p), ("d_feat_std", C.c_void_p),
                ("out_mean", C.c_float * 2), ("out_std", C.c_float * 2), ("feat_steps", C.c_int),
                ("l_min", C.c_int), ("l_max", C.c_int), ("window", C.c_int), ("accept_tol", C.c_double),
                ("t_min", C.c_double), ("t_max", C.c_double), ("fallback_rule", C.c_int),
                ("z_max", C.c_double)]


class Timings(C.Structure):
    _fields_ = [("assemble_ms", C.c_double), ("gkb_ms", C.c_double), ("svd_ms", C.c_double),
                ("select_ms", C.c_double), ("lift_ms", C.c_double), ("evaluate_ms", C.c_double),
                ("gkb_steps", C.c_int)]


EXPORTS = {
    "rbf_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.POINTER(Options)]),
    "rbf_destroy": (C.c_int, [C.c_void_p]),
    "rbf_last_error": (C.c_char_p, [C.c_void_p]),
    "rbf_workspace_bytes": (C.c_size_t, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int]),
    "rbf_get_timings": (C.c_int, [C.c_void_p, C.POINTER(Timings)]),
    "rbf_get_counters": (C.c_int, [C.c_void_p, C.POINTER(Counters), C.c_int]),
    "rbf_operator_init": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.c_void_p, C.c_int64, C.c_int64,
                                    C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                    C.c_int64]),
    "rbf_assemble": (C.c_int, [C.c_void_p, C.POINTER(Operator)]),
    "rbf_matvec": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.c_int, C.c_void_p, C.c_void_p]),
    "rbf_gkb": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.c_void_p, C.c_int, C.POINTER(GkbState)]),
    "rbf_gkb_resume": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.POINTER(GkbState), C.c_int]),
    "rbf_gkb_snapshot": (C.c_int, [C.c_void_p, C.POINTER(GkbState), C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    "rbf_gkb_restore": (C.c_int, [C.c_void_p, C.POINTER(GkbState), C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_int, C.c_int, C.c_double]),
    "rbf_gkb_many": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Operator), C.POINTER(C.c_void_p), C.c_int,
                               C.POINTER(GkbState), C.c_int, C.c_int]),
    "rbf_hkt_many": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(GkbState), C.c_int, C.c_double,
                               C.POINTER(C.c_void_p), C.POINTER(SolveInfo), C.c_int]),
    "rbf_projected_svd": (C.c_int, [C.c_void_p, C.POINTER(GkbState), C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int64]),
    "rbf_hkt": (C.c_int, [C.c_void_p, C.POINTER(GkbState), C.c_int, C.c_double, C.c_void_p,
                          C.c_void_p, C.POINTER(SolveInfo)]),
    "rbf_ine_tsvd": (C.c_int, [C.c_void_p, C.POINTER(GkbState), C.c_int, C.c_void_p, C.c_void_p,
                               C.POINTER(SolveInfo)]),
    "rbf_lsqr": (C.c_int, [C.c_void_p, C.POINTER(GkbState), C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                           C.POINTER(SolveInfo)]),
    "rbf_tikhonov": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.c_void_p, C.c_int, C.c_double,
                               C.c_void_p, C.POINTER(SolveInfo)]),
    "rbf_svd_full": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(C.c_int)]),
    "rbf_tsvd": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.c_void_p, C.c_int, C.c_void_p,
                           C.POINTER(SolveInfo)]),
    "rbf_evaluate": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.c_void_p, C.c_void_p, C.c_int64,
                               C.c_void_p]),
    "rbf_batch_gkb": (C.c_int, [C.c_void_p, C.POINTER(Batch), C.c_int, C.c_int]),
    "rbf_batch_hkt": (C.c_int, [C.c_void_p, C.POINTER(Batch), C.c_int, C.c_void_p, C.POINTER(C.c_double)]),
    "rbf_batch_evaluate": (C.c_int, [C.c_void_p, C.POINTER(Batch), C.c_int, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_int64), C.c_void_p]),
    "rbf_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(Tuning)]),
    "rbf_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "rbf_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                               C.POINTER(C.c_float)]),
    "rbf_mlp_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                               C.c_float]),
    "rbf_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float,
                                     C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_float)]),
    "rbf_stop_features": (C.c_int, [C.c_void_p, C.POINTER(GkbState), C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "rbf_evaluate_many": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.c_void_p, C.c_int64, C.c_int,
                                    C.c_void_p, C.c_int64, C.c_void_p]),
    "rbf_hkt_error_table": (C.c_int, [C.c_void_p, C.POINTER(GkbState), C.c_void_p, C.c_int64, C.c_int64,
                                      C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_void_p]),
    "rbf_learned_hkt": (C.c_int, [C.c_void_p, C.POINTER(Operator), C.c_void_p, C.POINTER(StopNet),
                                  C.POINTER(GkbState), C.c_void_p, C.c_void_p]),
    "rbf_batch_hkt_each": (C.c_int, [C.c_void_p, C.POINTER(Batch), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                     C.c_void_p, C.POINTER(C.c_double)]),
    "rbf_batch_learned_hkt": (C.c_int, [C.c_void_p, C.POINTER(Batch), C.POINTER(StopNet), C.c_void_p,
                                        C.c_void_p]),
    "rbf_matvec_t_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    "rbf_stopnet_init": (C.c_int, [C.c_void_p, C.POINTER(StopNet), C.c_void_p, C.POINTER(C.c_float),
                                   C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float),
                                   C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "rbf_stopnet_save": (C.c_int, [C.c_void_p, C.POINTER(StopNet), C.c_char_p]),
    "rbf_stopnet_load": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(StopNet), C.c_void_p]),
    "rbf_checked_build": (C.c_int, []),
    "rbf_check": (C.c_int, [C.c_void_p]),
    "rbf_check_selftest": (C.c_int, [C.c_void_p]),
    "rbf_probe_fp64": (C.c_int, [C.c_void_p, C.c_int, C.c_longlong, C.c_void_p, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
}

RBF_MLP_IN, RBF_MLP_HIDDEN, RBF_MLP_OUT = 20, 128, 2
RBF_MLP_PARAMS = 20 * 128 + 128 + 128 * 128 + 128 + 128 * 2 + 2
RBF_STOPNET_DEVICE_FLOATS = RBF_MLP_PARAMS + 2 * RBF_MLP_IN

RBF_NOALLOC_SCRATCH_DOUBLES = 1 << 20


def rbf_matvec_t_noalloc(A, lda, n, x, y, stream=None):
    """y = A^T x through the allocation-free entry point (no context)."""
    lib = load()
    s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    st = lib.rbf_matvec_t_noalloc(_ptr(A), lda, n, _ptr(x), _ptr(y), s)
    if st != RBF_OK:
        raise RbfError(st, "rbf_matvec_t_noalloc failed")

_lib = None


def load(path: str | None = None):
    """Load librbfkr.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    checked = os.environ.get("RBFKR_CHECKED", "") == "1"
    p = path or (_build.LIB_CHECKED if checked else LIB_PATH)
    if path is None:
        _build.build(checked=checked)
    if not os.path.exists(p):
        raise RuntimeError(f"librbfkr.so not found at {p}; the CUDA library is required")
    lib = C.CDLL(p)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_cuda:
            raise ValueError("device buffers must be CUDA tensors")
        if not t.is_contiguous():
            raise ValueError("device buffers must be contiguous")
        return t.data_ptr()
    return int(t)


class Context:
    """Owns one rbf_ctx.  Methods mirror the C entry points."""

    def __init__(self, device: int = 0, stream=None, timing: bool = False, **opts):
        self.lib = load()
        o = Options()
        for k, v in opts.items():
            setattr(o, k, v)
        o.timing = int(timing)
        self.grid_j = o.grid_j if o.grid_j > 0 else 321  # the library's default; 1 and 2 are rejected
        self.grid_t_lo, self.grid_t_hi = ((o.grid_t_lo, o.grid_t_hi) if o.grid_t_lo < o.grid_t_hi
                                          else (-16.0, 0.0))
        h = C.c_void_p()
        s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        st = self.lib.rbf_create(C.byref(h), device, s, C.byref(o))
        if st != RBF_OK:
            raise RbfError(st, "rbf_create failed")
        self.h = h

    def _check(self, st):
        if st != RBF_OK:
            raise RbfError(st, self.lib.rbf_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.rbf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- C entry points -------------------------------------------------
    def rbf_workspace_bytes(self, n, steps, storage, precision):
        return self.lib.rbf_workspace_bytes(self.h, n, steps, storage, precision)

    def rbf_get_timings(self):
        t = Timings()
        self._check(self.lib.rbf_get_timings(self.h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in Timings._fields_}

    def rbf_get_counters(self, reset=False):
        c = Counters()
        self._check(self.lib.rbf_get_counters(self.h, C.byref(c), 1 if reset else 0))
        return {"launches": c.launches, "product_launches": list(c.product_launches),
                "product_ms": list(c.product_ms), "product_busy_ms": c.product_busy_ms,
                "reorth_launches": c.reorth_launches, "reorth_ms": c.reorth_ms}

    def rbf_operator_init(self, nodes, n, n_interior, c, k, storage=RBF_ASSEMBLED, precision=RBF_FP64,
                          form=RBF_FORM_C, A=None, lda=0):
        op = Operator()
        self._check(self.lib.rbf_operator_init(self.h, C.byref(op), _ptr(nodes), n, n_interior, c, k,
                                               storage, precision, form, _ptr(A), lda))
        op._keep = (nodes, A)
        return op

    def rbf_assemble(self, op):
        self._check(self.lib.rbf_assemble(self.h, C.byref(op)))

    def rbf_matvec(self, op, trans, x, y):
        self._check(self.lib.rbf_matvec(self.h, C.byref(op), trans, _ptr(x), _ptr(y)))

    def rbf_gkb(self, op, f, steps, state):
        self._check(self.lib.rbf_gkb(self.h, C.byref(op), _ptr(f), steps, C.byref(state)))
        return state.steps_done

    def rbf_gkb_resume(self, op, state, more):
        self._check(self.lib.rbf_gkb_resume(self.h, C.byref(op), C.byref(state), more))
        return state.steps_done

    def rbf_gkb_snapshot(self, state):
        """Host checkpoint (numpy arrays) of a GKB state: W (l+1, n), Z (l, n), alpha, beta and scalars."""
        import numpy as np
        n, l = state.n, state.steps_done
        W = np.empty((l + 1, n))
        Z = np.empty((max(l, 1), n))
        al = np.empty(max(l, 1))
        be = np.empty(l + 1)
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        self._check(self.lib.rbf_gkb_snapshot(self.h, C.byref(state), p(W), p(Z), p(al), p(be)))
        return {"W": W, "Z": Z[:l], "alpha": al[:l], "beta": be, "steps_done": l, "breakdown": state.breakdown,
                "c_hat": state.c_hat}

    def rbf_gkb_restore(self, state, snap):
        import numpy as np
        arrs = [np.ascontiguousarray(snap[k], np.float64) for k in ("W", "Z", "alpha", "beta")]
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        self._check(self.lib.rbf_gkb_restore(self.h, C.byref(state), *[p(a) for a in arrs], int(snap["steps_done"]),
                                             int(snap["breakdown"]), float(snap["c_hat"])))

    def rbf_gkb_many(self, ops, fs, steps, states, lanes=0, assemble=False):
        """Independent GKB runs on the context's lanes; states are updated in place."""
        cnt = len(ops)
        if not (len(fs) == len(states) == cnt):
            raise ValueError("rbf_gkb_many: ops, fs and states must have the same length")
        op_arr = (Operator * cnt)(*ops)
        st_arr = (GkbState * cnt)(*states)
        f_arr = (C.c_void_p * cnt)(*[_ptr(f) for f in fs])
        st = self.lib.rbf_gkb_many(self.h, cnt, op_arr, f_arr, steps, st_arr, lanes, 1 if assemble else 0)
        for i in range(cnt):  # the C call wrote its copies: bring the host fields back
            for name in ("steps_done", "breakdown", "c_hat"):
                setattr(states[i], name, getattr(st_arr[i], name))
        self._check(st)
        return [s_.steps_done for s_ in states]

    def rbf_hkt_many(self, states, rule, lambda_in, coefs, lanes=0):
        cnt = len(states)
        st_arr = (GkbState * cnt)(*states)
        c_arr = (C.c_void_p * cnt)(*[_ptr(c) for c in coefs])
        infos = (SolveInfo * cnt)()
        self._check(self.lib.rbf_hkt_many(self.h, cnt, st_arr, rule, float(lambda_in), c_arr, infos, lanes))
        return list(infos)

    def rbf_stopnet_load(self, path, storage):
        """A stop network read by the library from a file written by rbf_stopnet_save;
        storage: float32 CUDA tensor of RBF_STOPNET_DEVICE_FLOATS (keep it alive)."""
        net = StopNet()
        self._check(self.lib.rbf_stopnet_load(self.h, os.fsencode(path), C.byref(net), _ptr(storage)))
        return net

    def rbf_stopnet_save(self, net, path):
        self._check(self.lib.rbf_stopnet_save(self.h, C.byref(net), os.fsencode(path)))

    def rbf_stopnet_init(self, storage, params, feat_mean, feat_std, out, rules, tols):
        import numpy as np
        net = StopNet()
        fp = lambda a: None if a is None else np.ascontiguousarray(a, np.float32).ctypes.data_as(C.POINTER(C.c_float))
        keep = [np.ascontiguousarray(a, np.float32) if a is not None else None for a in (params, feat_mean, feat_std, out)]
        r = (C.c_int * 4)(*[int(x) for x in rules])
        t = (C.c_double * 4)(*[float(x) for x in tols])
        self._check(self.lib.rbf_stopnet_init(self.h, C.byref(net), _ptr(storage), *[fp(a) for a in keep], r, t))
        return net

    def rbf_check(self):
        """Synchronise and report a failed device index check (bounds-checked build)."""
        self._check(self.lib.rbf_check(self.h))

    def rbf_check_selftest(self):
        self._check(self.lib.rbf_check_selftest(self.h))

    def rbf_probe_fp64(self, mode, iters, scratch):
        ms, flops = C.c_double(), C.c_double()
        self._check(self.lib.rbf_probe_fp64(self.h, mode, int(iters), _ptr(scratch), C.byref(ms), C.byref(flops)))
        return ms.value, flops.value

    def rbf_projected_svd(self, state, sigma, ftil, V, ldv):
        self._check(self.lib.rbf_projected_svd(self.h, C.byref(state), _ptr(sigma), _ptr(ftil),
                                               _ptr(V), ldv))

    @staticmethod
    def _curve_fits(curve, need, what):
        if curve is not None and hasattr(curve, "numel") and curve.numel() < need:
            raise ValueError(f"{what}: curve buffer holds {curve.numel()} values, needs {need}")

    def rbf_hkt(self, state, rule, lambda_in, coef, curve=None):
        self._curve_fits(curve, self.grid_j, "rbf_hkt")
        info = SolveInfo()
        self._check(self.lib.rbf_hkt(self.h, C.byref(state), rule, float(lambda_in), _ptr(coef),
                                     _ptr(curve), C.byref(info)))
        return info

    def rbf_ine_tsvd(self, state, rank, coef, curve=None):
        self._curve_fits(curve, state.steps_done, "rbf_ine_tsvd")
        info = SolveInfo()
        self._check(self.lib.rbf_ine_tsvd(self.h, C.byref(state), rank, _ptr(coef), _ptr(curve),
                                          C.byref(info)))
        return info

    def rbf_lsqr(self, state, rule, k_fixed, coef, curve=None):
        self._curve_fits(curve, state.steps_done, "rbf_lsqr")
        info = SolveInfo()
        self._check(self.lib.rbf_lsqr(self.h, C.byref(state), rule, int(k_fixed), _ptr(coef), _ptr(curve),
                                      C.byref(info)))
        return info

    def rbf_svd_full(self, op, sigma, f=None, fhat=None, V=None):
        sw = C.c_int(0)
        self._check(self.lib.rbf_svd_full(self.h, C.byref(op), _ptr(f), _ptr(sigma), _ptr(fhat), _ptr(V),
                                          C.byref(sw)))
        return sw.value

    def rbf_tsvd(self, op, f, rank, coef):
        info = SolveInfo()
        self._check(self.lib.rbf_tsvd(self.h, C.byref(op), _ptr(f), int(rank), _ptr(coef), C.byref(info)))
        return info

    def rbf_tikhonov(self, op, f, rule, lambda_in, coef):
        info = SolveInfo()
        self._check(self.lib.rbf_tikhonov(self.h, C.byref(op), _ptr(f), rule, float(lambda_in),
                                          _ptr(coef), C.byref(info)))
        return info

    def rbf_batch_gkb(self, batch, steps, form=RBF_FORM_C):
        self._check(self.lib.rbf_batch_gkb(self.h, C.byref(batch), steps, form))

    def rbf_batch_hkt(self, batch, rule, coef):
        lam = (C.c_double * batch.count)()
        self._check(self.lib.rbf_batch_hkt(self.h, C.byref(batch), rule, _ptr(coef), lam))
        return list(lam)

    def rbf_batch_evaluate(self, batch, coef, points, m, u, form=RBF_FORM_C):
        arr = (C.c_int64 * batch.count)(*m)
        self._check(self.lib.rbf_batch_evaluate(self.h, C.byref(batch), form, _ptr(coef), _ptr(points), arr,
                                                _ptr(u)))

    def rbf_batch_hkt_each(self, batch, rules, lambda_in, coef):
        B = batch.count
        r = (C.c_int * B)(*[int(x) for x in rules])
        li = (C.c_double * B)(*[float(x) for x in lambda_in])
        lam = (C.c_double * B)()
        self._check(self.lib.rbf_batch_hkt_each(self.h, C.byref(batch), r, li, _ptr(coef), lam))
        return list(lam)

    def rbf_batch_learned_hkt(self, batch, net, coef):
        infos = (LearnedInfo * batch.count)()
        self._check(self.lib.rbf_batch_learned_hkt(self.h, C.byref(batch), C.byref(net), _ptr(coef), infos))
        return list(infos)

    def rbf_get_tuning(self):
        t = Tuning()
        self._check(self.lib.rbf_get_tuning(self.h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def rbf_evaluate(self, op, coef, points, m, u):
        self._check(self.lib.rbf_evaluate(self.h, C.byref(op), _ptr(coef), _ptr(points), m, _ptr(u)))

    # --- learned stopping index and lambda --------------------------------
    def rbf_mlp_forward(self, params, x, batch, y):
        self._check(self.lib.rbf_mlp_forward(self.h, _ptr(params), _ptr(x), batch, _ptr(y)))

    def rbf_mlp_grad(self, params, x, t, batch, grad, want_loss=True):
        loss = C.c_float(0.0)
        self._check(self.lib.rbf_mlp_grad(self.h, _ptr(params), _ptr(x), _ptr(t), batch, _ptr(grad),
                                          C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def rbf_mlp_adam(self, params, m, v, grad, t, lr):
        self._check(self.lib.rbf_mlp_adam(self.h, _ptr(params), _ptr(m), _ptr(v), _ptr(grad), t, float(lr)))

    def rbf_mlp_train_step(self, params, m, v, t, lr, x, target, batch, grad, want_loss=False):
        loss = C.c_float(0.0)
        self._check(self.lib.rbf_mlp_train_step(self.h, _ptr(params), _ptr(m), _ptr(v), t, float(lr), _ptr(x),
                                                _ptr(target), batch, _ptr(grad),
                                                C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def rbf_stop_features(self, state, j, feat, mean=None, std=None):
        self._check(self.lib.rbf_stop_features(self.h, C.byref(state), j, _ptr(mean), _ptr(std), _ptr(feat)))

    def rbf_hkt_error_table(self, state, G, ldg, m, uref, ells, t_stride, err):
        arr = (C.c_int * len(ells))(*[int(x) for x in ells])
        self._check(self.lib.rbf_hkt_error_table(self.h, C.byref(state), _ptr(G), ldg, m, _ptr(uref), len(ells),
                                                 arr, t_stride, _ptr(err)))

    def rbf_learned_hkt(self, op, f, net, state, coef):
        info = LearnedInfo()
        self._check(self.lib.rbf_learned_hkt(self.h, C.byref(op), _ptr(f), C.byref(net), C.byref(state),
                                             _ptr(coef), C.byref(info)))
        return info

    def rbf_evaluate_many(self, op, coefs, ldc, ncoef, points, m, u):
        self._check(self.lib.rbf_evaluate_many(self.h, C.byref(op), _ptr(coefs), ldc, ncoef, _ptr(points), m,
                                               _ptr(u)))


def make_state(torch, n, capacity, device="cuda"):
    """Allocate caller-owned GKB buffers as torch tensors and wrap them."""
    ld = n
    W = torch.zeros((capacity + 1, ld), dtype=torch.float64, device=device)  # column j = W[j]
    Z = torch.zeros((capacity, ld), dtype=torch.float64, device=device)
    alpha = torch.zeros(capacity, dtype=torch.float64, device=device)
    beta = torch.zeros(capacity + 1, dtype=torch.float64, device=device)
    st = GkbState()
    st.d_W, st.ldw = W.data_ptr(), ld
    st.d_Z, st.ldz = Z.data_ptr(), ld
    st.d_alpha, st.d_beta = alpha.data_ptr(), beta.data_ptr()
    st.capacity, st.n = capacity, n
    st.steps_done, st.breakdown, st.c_hat = 0, 0, 0.0
    st._keep = (W, Z, alpha, beta)
    return st, W, Z, alpha, beta


def padded_lda(n, precision):
    """Leading dimension used for assembled matrices: a multiple of 32 elements."""
    return ((n + 31) // 32) * 32


def make_batch(torch, node_sets, cs, ks, fs, capacity, device="cuda"):
    """Concatenate instances into the rbf_batch layout (caller-owned torch buffers).

    node_sets: objects with .X (n x 3 float64) and .n_interior; fs: list of f_b.
    Returns (Batch, dict of tensors and host arrays); keep the dict alive.
    """
    import numpy as np
    B = len(node_sets)
    ns = [int(s.X.shape[0]) for s in node_sets]
    T = int(sum(ns))
    nodes = np.concatenate([np.ascontiguousarray(s.X.T).ravel() for s in node_sets])
    f = np.concatenate([np.asarray(x, dtype=np.float64) for x in fs])
    keep = {
        "nodes": torch.as_tensor(nodes, dtype=torch.float64, device=device),
        "f": torch.as_tensor(f, dtype=torch.float64, device=device),
        "W": torch.zeros((capacity + 1) * T, dtype=torch.float64, device=device),
        "Z": torch.zeros(capacity * T, dtype=torch.float64, device=device),
        "alpha": torch.zeros(B * capacity, dtype=torch.float64, device=device),
        "beta": torch.zeros(B * (capacity + 1), dtype=torch.float64, device=device),
        "n": (C.c_int64 * B)(*ns),
        "ni": (C.c_int64 * B)(*[int(s.n_interior) for s in node_sets]),
        "c": (C.c_double * B)(*[float(x) for x in cs]),
        "k": (C.c_double * B)(*[float(x) for x in ks]),
        "steps_done": (C.c_int * B)(),
        "breakdown": (C.c_int * B)(),
        "offsets": np.concatenate([[0], np.cumsum(ns)]).astype(np.int64),
    }
    bt = Batch()
    bt.count = B
    bt.n, bt.n_interior = keep["n"], keep["ni"]
    bt.c, bt.k = keep["c"], keep["k"]
    bt.d_nodes, bt.d_f = keep["nodes"].data_ptr(), keep["f"].data_ptr()
    bt.capacity = capacity
    bt.d_W, bt.d_Z = keep["W"].data_ptr(), keep["Z"].data_ptr()
    bt.d_alpha, bt.d_beta = keep["alpha"].data_ptr(), keep["beta"].data_ptr()
    bt.steps_done, bt.breakdown = keep["steps_done"], keep["breakdown"]
    return bt, keep
