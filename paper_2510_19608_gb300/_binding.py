"""ctypes binding of libokron (include/okron.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy/torch
arrays to the C structs and back.  Importing it does not build anything: call
``paper_2510_19608_gb300.build.build()`` first.  When the library is missing the
import of :func:`lib` raises -- there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ECUDA, EPF, ETIMEOUT, ENOTREADY, ESINGULAR, EINTERNAL = range(9)
SCORER_FEATURES = 14     # OKR_SCORER_FEATURES: floats per candidate row of okr_get_recorded_features
STATIC_MAX_BUS = 4096    # OKR_STATIC_MAX_BUS: largest feeder of okr_power_flow_static


class OkrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"okron status {status}: {msg}")
        self.status = status


class Feeder(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_scen", C.c_int32),
                ("parent", C.c_void_p), ("phases", C.c_void_p), ("z_line", C.c_void_p), ("s_load", C.c_void_p),
                ("v_slack", (C.c_double * 2) * 3)]


class Params(C.Structure):
    _fields_ = [("margin", C.c_double), ("target_reduction", C.c_double), ("tie_tol", C.c_double),
                ("objective", C.c_int32), ("precision", C.c_int32), ("record_iters", C.c_int32),
                ("max_merges", C.c_int32), ("profile", C.c_int32), ("scorer_topk", C.c_int32),
                ("engine", C.c_int32), ("max_spins", C.c_int64), ("prune_exact", C.c_int32),
                ("reserved", C.c_int32)]


class Summary(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_scen", C.c_int32), ("n_iter", C.c_int32), ("stop_reason", C.c_int32),
                ("pf_sweeps", C.c_int32), ("n_kept", C.c_int32), ("candidates", C.c_int64),
                ("smice", C.c_double), ("max_error", C.c_double), ("launches", C.c_int64),
                ("search_ms", C.c_double), ("sweeps", C.c_int64), ("sweep_ms", C.c_double), ("flops", C.c_double),
                ("rechecks", C.c_int32), ("recheck_cands", C.c_int32), ("phase_ms", C.c_double * 16),
                ("kron_ms", C.c_double), ("scorer_fallbacks", C.c_int32), ("inc_mismatches", C.c_int32),
                ("engine", C.c_int32), ("pad", C.c_int32), ("terms", C.c_int64),
                ("inc_threads", C.c_int32), ("inc_eval_warps", C.c_int32), ("inc_shared_entries", C.c_int32),
                ("inc_records", C.c_int32), ("pruned", C.c_int64)]


class IncShape(C.Structure):
    _fields_ = [("threads", C.c_int32), ("eval_warps", C.c_int32), ("shared_entries", C.c_int32),
                ("records", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_iter", C.c_int32), ("stop_reason", C.c_int32), ("n_kept", C.c_int32),
                ("candidates", C.c_int64), ("smice", C.c_double), ("max_error", C.c_double)]


class BatchStats(C.Structure):
    _fields_ = [("setup_ms", C.c_double), ("search_ms", C.c_double), ("candidates", C.c_int64),
                ("config", C.c_int32), ("ctas", C.c_int32), ("fallbacks", C.c_int32), ("reserved", C.c_int32)]


# okr_alloc_fn / okr_free_fn
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p)

EXPORTS = ("okr_default_params", "okr_create", "okr_destroy", "okr_status_str", "okr_last_error",
           "okr_reduce", "okr_reduce_device", "okr_reduce_ops", "okr_power_flow", "okr_get_summary",
           "okr_get_decisions", "okr_get_assignment", "okr_get_voltages", "okr_get_recorded",
           "okr_power_flow_static", "okr_kron", "okr_reduce_batch", "okr_batch_autotune",
           "okr_set_batch_config", "okr_radialize", "okr_get_recorded_features", "okr_scorer_init",
           "okr_scorer_params", "okr_scorer_gradient", "okr_scorer_train", "okr_scorer_predict",
           "okr_evaluate", "okr_scorer_predict_tc", "okr_batch_plan_create", "okr_batch_plan_run", "okr_batch_plan_set_loads",
           "okr_batch_plan_destroy", "okr_set_inc_shape", "okr_get_inc_shape",
           "okr_set_allocator", "okr_inc_autotune", "okr_result_take", "okr_result_free", "okr_result_summary",
           "okr_result_assignment", "okr_result_decisions", "okr_result_errors", "okr_result_ykron",
           "okr_result_stats")


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libokron.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise OSError(f"{path} is missing: build it with paper_2510_19608_gb300.build.build()")
            L = C.CDLL(path)
            P, I32 = C.c_void_p, C.c_int32
            L.okr_default_params.argtypes = [C.POINTER(Params)]
            L.okr_default_params.restype = None
            L.okr_create.argtypes = [C.POINTER(P), C.c_int, P]
            L.okr_destroy.argtypes = [P]
            L.okr_status_str.argtypes = [C.c_int]
            L.okr_status_str.restype = C.c_char_p
            L.okr_last_error.argtypes = [P]
            L.okr_last_error.restype = C.c_char_p
            for fn in ("okr_reduce", "okr_reduce_device"):
                getattr(L, fn).argtypes = [P, C.POINTER(Feeder), C.POINTER(Params)]
            L.okr_reduce_ops.argtypes = [P, C.POINTER(Feeder), P, P, C.POINTER(Params)]
            L.okr_power_flow.argtypes = [P, C.POINTER(Feeder), P, P, P]
            L.okr_power_flow_static.argtypes = [C.POINTER(Feeder), P, P, P, P]
            L.okr_kron.argtypes = [P, P, I32, P, P, P]
            L.okr_reduce_batch.argtypes = [P, I32, P, P, I32, P, P, P]
            L.okr_batch_autotune.argtypes = [P, I32, P, P, I32, P, P]
            L.okr_set_batch_config.argtypes = [P, I32]
            L.okr_batch_plan_create.argtypes = [P, I32, P, P, I32, C.POINTER(P)]
            L.okr_batch_plan_run.argtypes = [P, P, P, P]
            L.okr_batch_plan_set_loads.argtypes = [P, I32, P]
            L.okr_batch_plan_destroy.argtypes = [P]
            L.okr_batch_plan_destroy.restype = None
            L.okr_radialize.argtypes = [P, P, P, P]
            L.okr_get_recorded_features.argtypes = [P, I32, I32, P, P]
            L.okr_evaluate.argtypes = [P, C.POINTER(Feeder), P, P, P]
            L.okr_scorer_init.argtypes = [P, I32, P]
            L.okr_scorer_params.argtypes = [P, P, P]
            L.okr_scorer_gradient.argtypes = [P, P, P, I32, P, P]
            L.okr_scorer_train.argtypes = [P, P, P, C.c_int64, I32, I32, C.c_float, P]
            L.okr_scorer_predict.argtypes = [P, P, C.c_int64, P]
            L.okr_scorer_predict_tc.argtypes = [P, P, C.c_int64, P]
            L.okr_get_summary.argtypes = [P, C.POINTER(Summary)]
            L.okr_set_inc_shape.argtypes = [P, P]
            L.okr_set_allocator.argtypes = [P, ALLOC_FN, FREE_FN, P]
            L.okr_inc_autotune.argtypes = [P, I32, P, P, I32, C.POINTER(IncShape), P, P, I32, P]
            L.okr_result_take.argtypes = [P, I32, C.POINTER(P)]
            L.okr_result_free.argtypes = [P]
            L.okr_result_free.restype = None
            L.okr_result_summary.argtypes = [P, C.POINTER(Summary)]
            L.okr_result_assignment.argtypes = [P, P, P, P]
            L.okr_result_decisions.argtypes = [P, I32, P, P, P, P, P, P, P]
            L.okr_result_errors.argtypes = [P, P, P, P, P, P, P]
            L.okr_result_ykron.argtypes = [P, I32, P, P, P]
            L.okr_result_stats.argtypes = [P, P, P, P]
            L.okr_get_inc_shape.argtypes = [P, C.POINTER(IncShape)]
            L.okr_get_decisions.argtypes = [P, I32, P, P, P, P, P, P]
            L.okr_get_assignment.argtypes = [P, P]
            L.okr_get_voltages.argtypes = [P, P, P]
            L.okr_get_recorded.argtypes = [P, I32, I32, P, P, P, P, P]
            for fn in EXPORTS:
                if fn not in ("okr_default_params", "okr_status_str", "okr_last_error", "okr_batch_plan_destroy",
                              "okr_result_free"):
                    getattr(L, fn).restype = C.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def default_params(**over) -> Params:
    p = Params()
    lib().okr_default_params(C.byref(p))
    for k, v in over.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


class HostFeeder:
    """Keeps contiguous host copies alive while a call uses their pointers."""

    def __init__(self, feeder):
        self.parent = np.ascontiguousarray(feeder.parent, dtype=np.int32)
        self.phases = np.ascontiguousarray(feeder.phases, dtype=np.uint8)
        self.z_line = np.ascontiguousarray(feeder.z_line, dtype=np.float64)
        s = getattr(feeder, "s_load", None)
        self.s_load = None if s is None else np.ascontiguousarray(s, dtype=np.float64)
        self.v_slack = np.ascontiguousarray(feeder.v_slack, dtype=np.float64).reshape(3, 2)
        self.n_scen = int(self.s_load.shape[0]) if self.s_load is not None else int(getattr(feeder, "n_scen"))
        self.c = Feeder()
        self.c.n_bus = self.parent.shape[0]
        self.c.n_scen = self.n_scen
        self.c.parent = _ptr(self.parent).value
        self.c.phases = _ptr(self.phases).value
        self.c.z_line = _ptr(self.z_line).value
        self.c.s_load = None if self.s_load is None else _ptr(self.s_load).value
        for p in range(3):
            self.c.v_slack[p][0] = self.v_slack[p, 0]
            self.c.v_slack[p][1] = self.v_slack[p, 1]


def device_feeder(n_bus: int, n_scen: int, parent_ptr: int, phases_ptr: int, z_ptr: int, s_ptr: int,
                  v_slack) -> Feeder:
    """okr_feeder whose arrays are device pointers (e.g. torch tensor data_ptr())."""
    f = Feeder()
    f.n_bus, f.n_scen = int(n_bus), int(n_scen)
    f.parent, f.phases, f.z_line, f.s_load = int(parent_ptr), int(phases_ptr), int(z_ptr), int(s_ptr)
    vs = np.asarray(v_slack, dtype=np.float64).reshape(3, 2)
    for p in range(3):
        f.v_slack[p][0], f.v_slack[p][1] = vs[p, 0], vs[p, 1]
    return f


def power_flow_static(dfeeder: Feeder, vhat_ptr: int, ihat_ptr: int | None = None, stream: int | None = None) -> int:
    """okr_power_flow_static: load flow into caller device buffers, no device allocation.

    dfeeder from device_feeder(); vhat_ptr / ihat_ptr: device addresses of
    [n_scen][n_bus][3][2] float64 buffers.  Returns the sweeps used; raises
    OkrError on a non-OK status.
    """
    sw = C.c_int32()
    st = lib().okr_power_flow_static(C.byref(dfeeder), C.c_void_p(int(vhat_ptr)),
                                     C.c_void_p(int(ihat_ptr)) if ihat_ptr else None, C.byref(sw),
                                     C.c_void_p(int(stream)) if stream else None)
    if st != OK:
        raise OkrError(st, lib().okr_status_str(st).decode())
    return int(sw.value)


class Context:
    """One okr_ctx: a CUDA stream and the device workspace."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self._h = C.c_void_p()
        self._check(lib().okr_create(C.byref(self._h), int(device), C.c_void_p(stream) if stream else None))
        self.n_bus = 0
        self.n_scen = 0

    def close(self):
        if self._h:
            lib().okr_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, status: int):
        if status != OK:
            h = getattr(self, "_h", None)
            msg = lib().okr_last_error(h).decode() if h else lib().okr_status_str(status).decode()
            raise OkrError(status, msg or lib().okr_status_str(status).decode())

    # ---- entry points
    def reduce(self, feeder, params: Params):
        hf = HostFeeder(feeder)
        self._check(lib().okr_reduce(self._h, C.byref(hf.c), C.byref(params)))
        self.n_bus, self.n_scen = hf.c.n_bus, hf.c.n_scen

    def reduce_device(self, dfeeder: Feeder, params: Params):
        self._check(lib().okr_reduce_device(self._h, C.byref(dfeeder), C.byref(params)))
        self.n_bus, self.n_scen = dfeeder.n_bus, dfeeder.n_scen

    def reduce_ops(self, feeder, vhat: np.ndarray, ihat: np.ndarray, params: Params):
        hf = HostFeeder(feeder)
        vh = np.ascontiguousarray(np.stack([vhat.real, vhat.imag], -1) if np.iscomplexobj(vhat) else vhat, dtype=np.float64)
        ih = np.ascontiguousarray(np.stack([ihat.real, ihat.imag], -1) if np.iscomplexobj(ihat) else ihat, dtype=np.float64)
        hf.c.n_scen = vh.shape[0]
        self._check(lib().okr_reduce_ops(self._h, C.byref(hf.c), _ptr(vh), _ptr(ih), C.byref(params)))
        self.n_bus, self.n_scen = hf.c.n_bus, hf.c.n_scen

    def power_flow(self, feeder):
        hf = HostFeeder(feeder)
        n, L = hf.c.n_bus, hf.c.n_scen
        v = np.zeros((L, n, 3, 2))
        i = np.zeros((L, n, 3, 2))
        sw = C.c_int32()
        self._check(lib().okr_power_flow(self._h, C.byref(hf.c), _ptr(v), _ptr(i), C.byref(sw)))
        return v[..., 0] + 1j * v[..., 1], i[..., 0] + 1j * i[..., 1], int(sw.value)

    @staticmethod
    def _batch_args(feeders, params):
        hfs = [HostFeeder(f) for f in feeders]
        arr = (Feeder * len(hfs))(*[h.c for h in hfs])
        plist = params if isinstance(params, (list, tuple)) else [params]
        parr = (Params * len(plist))(*plist)
        return hfs, arr, parr, len(plist)

    def reduce_batch(self, feeders, params, want_assignment=True):
        """okr_reduce_batch: many feeders in one launch.  params: one Params or
        one per feeder.  Returns (items, assignments or None, stats) with items
        and stats as dicts and one int32 array per feeder."""
        hfs, arr, parr, npar = self._batch_args(feeders, params)
        nf = len(hfs)
        items = (BatchItem * nf)()
        st = BatchStats()
        tot = sum(h.c.n_bus for h in hfs)
        sup = np.zeros(tot, np.int32) if want_assignment else None
        self._check(lib().okr_reduce_batch(self._h, nf, arr, parr, npar, items,
                                           _ptr(sup) if sup is not None else None, C.byref(st)))
        out = [{k: getattr(it, k) for k, _ in BatchItem._fields_} for it in items]
        parts = None
        if sup is not None:
            parts, o = [], 0
            for h in hfs:
                parts.append(sup[o:o + h.c.n_bus].copy())
                o += h.c.n_bus
        return out, parts, {k: getattr(st, k) for k, _ in BatchStats._fields_}

    def batch_plan(self, feeders, params):
        """okr_batch_plan_create: the batch staged once and captured as one CUDA
        graph; run() replays it."""
        return BatchPlan(self, feeders, params)

    def set_allocator(self, alloc=None, free=None):
        """okr_set_allocator: alloc(bytes, device, stream) -> int device address
        (0 on failure) and free(ptr, device, stream), called for every device
        block of this context; None, None restores cudaMalloc / cudaFree.  Call
        right after creating the context."""
        if alloc is None and free is None:
            self._alloc_cbs = None
            self._check(lib().okr_set_allocator(self._h, ALLOC_FN(), FREE_FN(), None))
            return

        def _a(user, nbytes, device, stream):
            try:
                return int(alloc(int(nbytes), int(device), int(stream or 0))) or None
            except Exception:
                return None

        def _f(user, ptr, device, stream):
            try:
                free(int(ptr), int(device), int(stream or 0))
            except Exception:
                pass

        cbs = (ALLOC_FN(_a), FREE_FN(_f))
        self._check(lib().okr_set_allocator(self._h, cbs[0], cbs[1], None))
        self._alloc_cbs = cbs             # the library calls them until the context is closed

    def use_torch_allocator(self):
        """Device memory from torch's caching allocator (torch.cuda.caching_allocator_alloc
        on the context's device and stream)."""
        import torch

        def alloc(nbytes, device, stream):
            return torch.cuda.caching_allocator_alloc(nbytes, device, stream)

        def free(ptr, device, stream):
            torch.cuda.caching_allocator_delete(ptr)

        self.set_allocator(alloc, free)

    def set_inc_shape(self, threads: int = 0, eval_warps: int = 0, shared_entries: int = 0, records: int = 0):
        """okr_set_inc_shape: launch shape of the incremental engine (0 = default)."""
        sh = IncShape(int(threads), int(eval_warps), int(shared_entries), int(records))
        self._check(lib().okr_set_inc_shape(self._h, C.byref(sh)))

    def reset_inc_shape(self):
        """okr_set_inc_shape(NULL): every field back to its default."""
        self._check(lib().okr_set_inc_shape(self._h, None))

    def inc_shape(self) -> dict:
        """okr_get_inc_shape: the context's shape, defaults filled in."""
        sh = IncShape()
        self._check(lib().okr_get_inc_shape(self._h, C.byref(sh)))
        return {k: getattr(sh, k) for k, _ in IncShape._fields_}

    def inc_autotune(self, feeders, params):
        """okr_inc_autotune: times the incremental engine's shapes on one feeder
        (a list of one) or a batch; keeps the fastest.  Returns (best shape,
        [(shape, search ms), ...])."""
        hfs, arr, parr, npar = self._batch_args(feeders, params)
        cap = 32
        best = IncShape()
        shapes = (IncShape * cap)()
        ms = (C.c_double * cap)()
        cnt = C.c_int32()
        self._check(lib().okr_inc_autotune(self._h, len(hfs), arr, parr, npar, C.byref(best), shapes, ms, cap,
                                           C.byref(cnt)))
        self.n_bus, self.n_scen = hfs[0].c.n_bus, hfs[0].c.n_scen
        as_dict = lambda sh: {k: getattr(sh, k) for k, _ in IncShape._fields_}   # noqa: E731
        return as_dict(best), [(as_dict(shapes[i]), ms[i]) for i in range(min(cnt.value, cap))]

    def set_batch_config(self, config: int):
        """okr_set_batch_config: team shape 0/1/2/3 = 1/2/4/8 CTAs per feeder."""
        self._check(lib().okr_set_batch_config(self._h, int(config)))

    def batch_autotune(self, feeders, params):
        """okr_batch_autotune: returns (best config, search ms per config)."""
        hfs, arr, parr, npar = self._batch_args(feeders, params)
        cfg = C.c_int32()
        ms = (C.c_double * 4)()
        self._check(lib().okr_batch_autotune(self._h, len(hfs), arr, parr, npar, C.byref(cfg), ms))
        return int(cfg.value), list(ms)

    def radialize(self, kept=None):
        """okr_radialize: critical-bus flags (caller order) of `kept` (None = the
        last reduction's super-nodes)."""
        n = int(self.summary()["n_bus"]) if kept is None else len(kept)
        kp = None if kept is None else np.ascontiguousarray(kept, dtype=np.uint8)
        out = np.zeros(n, np.uint8)
        cnt = C.c_int32()
        self._check(lib().okr_radialize(self._h, _ptr(kp) if kp is not None else None, _ptr(out), C.byref(cnt)))
        assert int(cnt.value) == int(out.sum())
        return out

    def evaluate(self, feeder, super_of):
        """okr_evaluate: (max error per scenario, reduced voltages [L, n, 3] complex)."""
        hf = HostFeeder(feeder)
        sup = np.ascontiguousarray(super_of, dtype=np.int32)
        L, n = hf.c.n_scen, hf.c.n_bus
        err = np.zeros(L)
        v = np.zeros((L, n, 3, 2))
        self._check(lib().okr_evaluate(self._h, C.byref(hf.c), _ptr(sup), _ptr(err), _ptr(v)))
        return err, v[..., 0] + 1j * v[..., 1]

    # ---- learned scorer
    def recorded_features(self, it: int) -> np.ndarray:
        cnt = C.c_int32()
        self._check(lib().okr_get_recorded_features(self._h, it, 0, None, C.byref(cnt)))
        out = np.zeros((int(cnt.value), SCORER_FEATURES), np.float32)
        self._check(lib().okr_get_recorded_features(self._h, it, out.shape[0], _ptr(out), C.byref(cnt)))
        return out

    def scorer_init(self, n_features: int, theta=None):
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
        self._check(lib().okr_scorer_init(self._h, int(n_features), _ptr(th) if th is not None else None))

    def scorer_params(self) -> np.ndarray:
        k = C.c_int32()
        self._check(lib().okr_scorer_params(self._h, None, C.byref(k)))
        out = np.zeros(int(k.value), np.float32)
        self._check(lib().okr_scorer_params(self._h, _ptr(out), C.byref(k)))
        return out

    def scorer_gradient(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(self.scorer_params().size, np.float32)
        loss = C.c_double()
        self._check(lib().okr_scorer_gradient(self._h, _ptr(x), _ptr(t), int(x.shape[0]), _ptr(g), C.byref(loss)))
        return g, float(loss.value)

    def scorer_train(self, x, t, batch: int, epochs: int, lr: float) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        el = np.zeros(max(epochs, 1))
        self._check(lib().okr_scorer_train(self._h, _ptr(x), _ptr(t), int(x.shape[0]), int(batch), int(epochs),
                                           float(lr), _ptr(el)))
        return el[:epochs]

    def scorer_predict(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros(x.shape[0], np.float32)
        self._check(lib().okr_scorer_predict(self._h, _ptr(x), int(x.shape[0]), _ptr(y)))
        return y

    def scorer_predict_tc(self, x) -> np.ndarray:
        """okr_scorer_predict_tc: the same network on the tensor cores (bfloat16
        layer inputs, FP32 accumulation)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros(x.shape[0], np.float32)
        self._check(lib().okr_scorer_predict_tc(self._h, _ptr(x), int(x.shape[0]), _ptr(y)))
        return y

    def kron(self, kept=None):
        """Y_Kron onto `kept` (caller-order flags; None = the last reduction's
        super-nodes).  Returns (Y complex [k, k], phase_node int32 [k])."""
        kp = None
        if kept is not None:
            kp = np.ascontiguousarray(kept, dtype=np.uint8)
        k = C.c_int32()
        self._check(lib().okr_kron(self._h, _ptr(kp) if kp is not None else None, 0, None, None, C.byref(k)))
        K = int(k.value)
        y = np.zeros((K, K, 2))
        pn = np.zeros(K, np.int32)
        self._check(lib().okr_kron(self._h, _ptr(kp) if kp is not None else None, K, _ptr(y), _ptr(pn), C.byref(k)))
        return y[..., 0] + 1j * y[..., 1], pn

    def take_result(self, with_ykron: bool = False) -> "Result":
        """okr_result_take: the last reduction's results as a library-owned object."""
        h = C.c_void_p()
        self._check(lib().okr_result_take(self._h, 1 if with_ykron else 0, C.byref(h)))
        return Result(h)

    # ---- results
    def summary(self) -> dict:
        s = Summary()
        self._check(lib().okr_get_summary(self._h, C.byref(s)))
        out = {k: getattr(s, k) for k, _ in Summary._fields_}
        out["phase_ms"] = list(s.phase_ms)
        return out

    def decisions(self) -> dict:
        t = self.summary()["n_iter"]
        cap = max(t, 1)
        s = np.zeros(cap, np.int32)
        r = np.zeros(cap, np.int32)
        sm = np.zeros(cap)
        me = np.zeros(cap)
        gap = np.zeros(cap)
        nc = np.zeros(cap, np.int32)
        self._check(lib().okr_get_decisions(self._h, cap, _ptr(s), _ptr(r), _ptr(sm), _ptr(me), _ptr(gap), _ptr(nc)))
        return dict(s=s[:t], r=r[:t], score=sm[:t], maxerr=me[:t], gap=gap[:t], ncand=nc[:t])

    def assignment(self) -> np.ndarray:
        out = np.zeros(self.n_bus, np.int32)
        self._check(lib().okr_get_assignment(self._h, _ptr(out)))
        return out

    def voltages(self):
        v = np.zeros((self.n_scen, self.n_bus, 3, 2))
        w = np.zeros((self.n_scen, self.n_bus, 3, 2))
        self._check(lib().okr_get_voltages(self._h, _ptr(v), _ptr(w)))
        return v[..., 0] + 1j * v[..., 1], w[..., 0] + 1j * w[..., 1]

    def recorded(self, it: int) -> dict:
        cap = 2 * self.n_bus
        s = np.zeros(cap, np.int32)
        r = np.zeros(cap, np.int32)
        sc = np.zeros(cap)
        bd = np.zeros(cap)
        cnt = C.c_int32()
        self._check(lib().okr_get_recorded(self._h, int(it), cap, _ptr(s), _ptr(r), _ptr(sc), _ptr(bd), C.byref(cnt)))
        c = min(cnt.value, cap)
        return dict(s=s[:c], r=r[:c], score=sc[:c], bound=bd[:c])


class BatchPlan:
    """A batch of feeders captured as one CUDA graph (okr_batch_plan_*)."""

    def __init__(self, ctx: Context, feeders, params):
        self._ctx = ctx
        hfs, arr, parr, npar = ctx._batch_args(feeders, params)
        self._n = [h.c.n_bus for h in hfs]
        self._shapes = [(h.c.n_scen, h.c.n_bus) for h in hfs]
        h = C.c_void_p()
        ctx._check(lib().okr_batch_plan_create(ctx._h, len(hfs), arr, parr, npar, C.byref(h)))
        self._h = h

    def run(self, want_assignment=True):
        """okr_batch_plan_run: (items, assignments or None, stats) as Context.reduce_batch."""
        nf = len(self._n)
        items = (BatchItem * nf)()
        st = BatchStats()
        sup = np.zeros(sum(self._n), np.int32) if want_assignment else None
        self._ctx._check(lib().okr_batch_plan_run(self._h, items, _ptr(sup) if sup is not None else None,
                                                   C.byref(st)))
        out = [{k: getattr(it, k) for k, _ in BatchItem._fields_} for it in items]
        parts = None
        if sup is not None:
            parts, o = [], 0
            for n in self._n:
                parts.append(sup[o:o + n].copy())
                o += n
        return out, parts, {k: getattr(st, k) for k, _ in BatchStats._fields_}

    def set_loads(self, feeder: int, s_load):
        """okr_batch_plan_set_loads: feeder's loads for the following runs."""
        L, n = self._shapes[feeder]
        a = np.ascontiguousarray(s_load, dtype=np.float64)
        if a.shape != (L, n, 3, 2):
            raise ValueError(f"s_load must have shape {(L, n, 3, 2)}")
        self._ctx._check(lib().okr_batch_plan_set_loads(self._h, int(feeder), _ptr(a)))

    def close(self):
        if self._h:
            lib().okr_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _checked(status: int):
    if status != OK:
        raise OkrError(status, lib().okr_status_str(status).decode())


class Result:
    """An okr_result: one reduction's results, owned by the library until close()."""

    def __init__(self, handle):
        self._h = handle

    def close(self):
        if self._h:
            lib().okr_result_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def summary(self) -> dict:
        s = Summary()
        _checked(lib().okr_result_summary(self._h, C.byref(s)))
        out = {k: getattr(s, k) for k, _ in Summary._fields_}
        out["phase_ms"] = list(s.phase_ms)
        return out

    def assignment(self) -> np.ndarray:
        n, k = C.c_int32(), C.c_int32()
        _checked(lib().okr_result_assignment(self._h, None, C.byref(n), C.byref(k)))
        out = np.zeros(int(n.value), np.int32)
        _checked(lib().okr_result_assignment(self._h, _ptr(out), C.byref(n), C.byref(k)))
        return out

    def decisions(self) -> dict:
        cnt = C.c_int32()
        _checked(lib().okr_result_decisions(self._h, 0, None, None, None, None, None, None, C.byref(cnt)))
        t = int(cnt.value)
        cap = max(t, 1)
        s, r, nc = (np.zeros(cap, np.int32) for _ in range(3))
        sm, me, gap = (np.zeros(cap) for _ in range(3))
        _checked(lib().okr_result_decisions(self._h, cap, _ptr(s), _ptr(r), _ptr(sm), _ptr(me), _ptr(gap), _ptr(nc),
                                            C.byref(cnt)))
        return dict(s=s[:t], r=r[:t], score=sm[:t], maxerr=me[:t], gap=gap[:t], ncand=nc[:t])

    def errors(self) -> dict:
        me, sm = C.c_double(), C.c_double()
        L, n = C.c_int32(), C.c_int32()
        _checked(lib().okr_result_errors(self._h, C.byref(me), C.byref(sm), None, None, C.byref(L), C.byref(n)))
        vh = np.zeros((L.value, n.value, 3, 2))
        vr = np.zeros((L.value, n.value, 3, 2))
        _checked(lib().okr_result_errors(self._h, None, None, _ptr(vh), _ptr(vr), None, None))
        return dict(max_error=me.value, smice=sm.value, vhat=vh[..., 0] + 1j * vh[..., 1],
                    vred=vr[..., 0] + 1j * vr[..., 1])

    def ykron(self):
        k = C.c_int32()
        _checked(lib().okr_result_ykron(self._h, 0, None, None, C.byref(k)))
        K = int(k.value)
        y = np.zeros((K, K, 2))
        pn = np.zeros(K, np.int32)
        _checked(lib().okr_result_ykron(self._h, K, _ptr(y), _ptr(pn), C.byref(k)))
        return y[..., 0] + 1j * y[..., 1], pn

    def stats(self) -> dict:
        c, it, sec = C.c_int64(), C.c_int32(), C.c_double()
        _checked(lib().okr_result_stats(self._h, C.byref(c), C.byref(it), C.byref(sec)))
        return dict(candidates=c.value, iterations=it.value, seconds=sec.value)
