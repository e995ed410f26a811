"""ctypes binding of the C ABI in ``include/de.h`` (``libde_gb300.so``).

Argument marshalling only: every step of the DE generation runs in the
library's CUDA kernels.  The functions keep the C names (``de_init``,
``de_step``, ``de_run``, ``de_eval`` ...); each raises ``DEError`` when the
library returns a status other than ``DE_OK``.  Importing this module never
falls back to anything: if the shared library is missing it raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

DE_OK, DE_ERR_INVALID_ARG, DE_ERR_CUDA, DE_ERR_OOM, DE_ERR_TIMEOUT = 0, 1, 2, 3, 4
DE_ERR_NONFINITE, DE_ERR_STATE, DE_ERR_IO, DE_ERR_UNSUPPORTED = 5, 6, 7, 8
DE_OBJ_SPHERE, DE_OBJ_RASTRIGIN, DE_OBJ_ROSENBROCK, DE_OBJ_ACKLEY, DE_OBJ_ODE = 0, 1, 2, 3, 4
DE_OBJ_ZAKHAROV, DE_OBJ_SCHWEFEL, DE_OBJ_BENT_CIGAR, DE_OBJ_HGBAT, DE_OBJ_SCHAFFER_F6 = 5, 6, 7, 8, 9
DE_OBJ_KATSUURA, DE_OBJ_HAPPYCAT, DE_OBJ_GRIEWANK_ROSENBROCK, DE_OBJ_ELLIPTIC, DE_OBJ_GRIEWANK = 10, 11, 12, 13, 14
DE_OBJ_HYBRID1, DE_OBJ_HYBRID2, DE_OBJ_HYBRID3 = 15, 16, 17
DE_OBJ_COMPOSITION1, DE_OBJ_COMPOSITION2, DE_OBJ_COMPOSITION3 = 18, 19, 20
DE_PREC_FP64, DE_PREC_BF16X3, DE_PREC_TF32X3 = 0, 1, 2
DE_STOP_NONE, DE_STOP_TARGET, DE_STOP_EVALS, DE_STOP_GENERATIONS = 0, 1, 2, 3
DE_BAND_NEAR, DE_BAND_ALL = 0, 1
DE_RAND1BIN, DE_BEST1BIN, DE_RAND1EXP = 0, 1, 2
DE_MIGRATE_SYNC, DE_MIGRATE_ASYNC = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_int64)


class de_config(ctypes.Structure):
    _fields_ = [("np", ctypes.c_int32), ("d", ctypes.c_int32), ("f", ctypes.c_double), ("cr", ctypes.c_double),
                ("lo", ctypes.c_double), ("hi", ctypes.c_double), ("objective", ctypes.c_int32),
                ("scale", ctypes.c_double), ("shift", _dp), ("rot", _dp), ("seed", ctypes.c_uint64),
                ("run_id", ctypes.c_uint32), ("precision", ctypes.c_int32), ("target_error", ctypes.c_double),
                ("max_evals", ctypes.c_int64), ("max_generations", ctypes.c_int64),
                ("debug_capture", ctypes.c_int32), ("fp64_band", ctypes.c_int32), ("surrogate_k", ctypes.c_int32),
                ("surrogate_steps", ctypes.c_int32), ("strategy", ctypes.c_int32), ("jde", ctypes.c_int32),
                ("perm", _i32p)]


class de_result(ctypes.Structure):
    _fields_ = [("best_f", ctypes.c_double), ("best_index", ctypes.c_int32), ("stop_reason", ctypes.c_int32),
                ("generations", ctypes.c_int64), ("evals", ctypes.c_int64), ("seconds", ctypes.c_double)]


class de_debug(ctypes.Structure):
    _fields_ = [("idx", _i32p), ("jrand", _i32p), ("mask", _u32p), ("trial", _dp), ("f_trial", _dp),
                ("accept", _u8p), ("fp64_checked", _u8p), ("cand", _i32p)]


class DEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libde_gb300.so (building it first when it is missing or stale and
    nvcc is present).  Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing:
            try:
                path = _build.build()
            except RuntimeError:
                if not os.path.exists(path):
                    raise
        if not os.path.exists(path):
            raise OSError(f"libde_gb300.so is missing at {path}; run paper_2405_16551_gb300/build.py")
        lib = ctypes.CDLL(path)
        H = ctypes.c_void_p
        sigs = {
            "de_version": ([], ctypes.c_char_p),
            "de_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "de_last_error": ([H], ctypes.c_char_p),
            "de_init": ([ctypes.POINTER(de_config), ctypes.c_void_p, ctypes.POINTER(H)], ctypes.c_int),
            "de_init_batch": ([ctypes.POINTER(de_config), ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(H)],
                              ctypes.c_int),
            "de_step": ([H, ctypes.c_int64], ctypes.c_int),
            "de_reset": ([H, ctypes.c_int32], ctypes.c_int),
            "de_run": ([H, ctypes.POINTER(de_result)], ctypes.c_int),
            "de_eval": ([H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p],
                        ctypes.c_int),
            "de_get_population": ([H, ctypes.c_int32, _dp, _dp], ctypes.c_int),
            "de_set_population": ([H, ctypes.c_int32, _dp, _dp], ctypes.c_int),
            "de_set_generation": ([H, ctypes.c_int32, ctypes.c_int64], ctypes.c_int),
            "de_get_best": ([H, ctypes.c_int32, _dp, _i32p, _dp, _i64p, _i64p, _i32p], ctypes.c_int),
            "de_get_debug": ([H, ctypes.c_int32, ctypes.POINTER(de_debug)], ctypes.c_int),
            "de_get_shape": ([H, ctypes.c_int32, _i32p, _i32p, _i32p], ctypes.c_int),
            "de_get_stats": ([H, ctypes.c_int32, _i64p, _i64p], ctypes.c_int),
            "de_get_plan": ([H, _i32p, _i32p], ctypes.c_int),
            "de_save": ([H, ctypes.c_char_p], ctypes.c_int),
            "de_load": ([H, ctypes.c_char_p], ctypes.c_int),
            "de_destroy": ([H], ctypes.c_int),
            "de_get_surrogate_stats": ([H, _i64p, _i64p, _dp, _i32p], ctypes.c_int),
            "de_get_adaptive": ([H, ctypes.c_int32, _dp, _dp], ctypes.c_int),
            "de_selftest_f32_rounding": ([_dp, ctypes.c_int64], ctypes.c_int64),
            "de_selftest_fp64_rate": ([], ctypes.c_double),
            "de_init_islands": ([ctypes.POINTER(de_config), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.POINTER(H)], ctypes.c_int),
            "de_init_islands_ex": ([ctypes.POINTER(de_config), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(H)], ctypes.c_int),
            "de_set_adaptive": ([H, ctypes.c_int32, _dp, _dp], ctypes.c_int),
            "de_mlp_create": ([ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(H)], ctypes.c_int),
            "de_mlp_destroy": ([H], ctypes.c_int),
            "de_mlp_set_params": ([H, _fp], ctypes.c_int),
            "de_mlp_get_params": ([H, _fp], ctypes.c_int),
            "de_mlp_forward": ([H, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p], ctypes.c_int),
            "de_mlp_grad": ([H, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, _fp, _fp], ctypes.c_int),
            "de_mlp_train": ([H, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_float, _fp], ctypes.c_int),
            "de_eval_noalloc": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.c_void_p], ctypes.c_int),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def exported_symbols():
    return ["de_version", "de_status_string", "de_last_error", "de_init", "de_init_batch", "de_reset", "de_step", "de_run",
            "de_eval", "de_get_population", "de_set_population", "de_set_generation", "de_get_best",
            "de_get_debug", "de_get_shape", "de_get_stats", "de_get_plan", "de_save", "de_load", "de_destroy",
            "de_eval_noalloc", "de_mlp_create", "de_mlp_destroy", "de_mlp_set_params", "de_mlp_get_params",
            "de_mlp_forward", "de_mlp_grad", "de_mlp_train", "de_get_surrogate_stats", "de_get_adaptive",
            "de_set_adaptive", "de_init_islands", "de_init_islands_ex", "de_selftest_f32_rounding",
            "de_selftest_fp64_rate"]


def _status_name(s):
    try:
        return load().de_status_string(s).decode()
    except Exception:  # pragma: no cover - only for messages
        return f"status {s}"


def _check(status, h=None):
    if status != DE_OK:
        msg = load().de_last_error(h).decode()
        raise DEError(status, msg)


def _p(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


# ----------------------------------------------------------------------------- the C calls
def de_version() -> str:
    return load().de_version().decode()


def make_config(np_, d, f=0.5, cr=0.9, lo=-100.0, hi=100.0, objective=DE_OBJ_SPHERE, scale=1.0, shift=None,
                rot=None, seed=1, run_id=0, precision=DE_PREC_FP64, target_error=1e-8, max_evals=0,
                max_generations=1000, debug_capture=False, fp64_band=DE_BAND_NEAR, surrogate_k=0,
                surrogate_steps=0, strategy=DE_RAND1BIN, jde=False, perm=None):
    """A de_config; the returned object keeps the shift/rotation arrays alive."""
    c = de_config()
    c.np, c.d, c.f, c.cr, c.lo, c.hi = np_, d, f, cr, lo, hi
    c.objective, c.scale, c.seed, c.run_id, c.precision = objective, scale, seed, run_id, precision
    c.target_error, c.max_evals, c.max_generations = target_error, max_evals, max_generations
    c.debug_capture = 1 if debug_capture else 0
    c.fp64_band = fp64_band
    c.surrogate_k, c.surrogate_steps = surrogate_k, surrogate_steps
    c.strategy, c.jde = strategy, 1 if jde else 0
    keep = []
    if shift is not None:
        s = np.ascontiguousarray(shift, dtype=np.float64)
        keep.append(s)
        c.shift = _p(s)
    if rot is not None:
        m = np.ascontiguousarray(rot, dtype=np.float64)
        keep.append(m)
        c.rot = _p(m)
    if perm is not None:
        pm = np.ascontiguousarray(perm, dtype=np.int32)
        keep.append(pm)
        c.perm = _p(pm, _i32p)
    c._keep = keep
    return c


def de_init(cfg: de_config, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load().de_init(ctypes.byref(cfg), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h.value


def de_init_batch(cfgs, stream=None) -> int:
    arr = (de_config * len(cfgs))(*cfgs)
    h = ctypes.c_void_p()
    _check(load().de_init_batch(arr, len(cfgs), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h.value


def de_reset(h, run: int = -1):
    _check(load().de_reset(h, run), h)


def de_step(h, generations: int):
    _check(load().de_step(h, generations), h)


def de_run(h, nruns: int = 1):
    res = (de_result * nruns)()
    _check(load().de_run(h, res), h)
    return [dict(best_f=r.best_f, best_index=r.best_index, stop_reason=r.stop_reason, generations=r.generations,
                 evals=r.evals, seconds=r.seconds) for r in res]


def de_eval(h, run: int, x_dev_ptr: int, ld: int, n: int, f_dev_ptr: int):
    _check(load().de_eval(h, run, ctypes.c_void_p(x_dev_ptr), ld, n, ctypes.c_void_p(f_dev_ptr)), h)


def de_eval_noalloc(precision: int, objective: int, d: int, scale: float, shift_dev_ptr, rot_dev_ptr, x_dev_ptr: int,
                    ld: int, n: int, f_dev_ptr: int, stream=None):
    """Handle-free split-precision evaluation through the library's static
    scratch (no allocation); pointers are device addresses (ints), shift and
    rotation may be None."""
    st = load().de_eval_noalloc(precision, objective, d, scale, ctypes.c_void_p(shift_dev_ptr),
                                ctypes.c_void_p(rot_dev_ptr), ctypes.c_void_p(x_dev_ptr), ld, n,
                                ctypes.c_void_p(f_dev_ptr), ctypes.c_void_p(stream))
    _check(st, None)


# ----------------------------------------------------------------------------- surrogate network
DE_MLP_PARAMS = 71425
MLP_SHAPES = (("W1", (256, 20)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("w3", (256,)), ("b3", (1,)))


def mlp_unpack(p):
    """Parameter vector -> dict of arrays (float64 copies)."""
    out, off = {}, 0
    for k, shp in MLP_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(p[off:off + n], dtype=np.float64).reshape(shp).copy()
        off += n
    return out


def mlp_pack(d):
    return np.concatenate([np.asarray(d[k], dtype=np.float32).ravel() for k, _ in MLP_SHAPES])


def de_mlp_create(seed=1, stream=None):
    h = ctypes.c_void_p()
    _check(load().de_mlp_create(seed, stream, ctypes.byref(h)), None)
    return h.value


def de_mlp_destroy(m):
    load().de_mlp_destroy(m)


def de_mlp_set_params(m, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == DE_MLP_PARAMS
    _check(load().de_mlp_set_params(m, p.ctypes.data_as(_fp)), None)


def de_mlp_get_params(m):
    p = np.zeros(DE_MLP_PARAMS, dtype=np.float32)
    _check(load().de_mlp_get_params(m, p.ctypes.data_as(_fp)), None)
    return p


def de_mlp_forward(m, x_dev_ptr: int, ld: int, n: int, y_dev_ptr: int):
    _check(load().de_mlp_forward(m, ctypes.c_void_p(x_dev_ptr), ld, n, ctypes.c_void_p(y_dev_ptr)), None)


def de_mlp_grad(m, x_dev_ptr: int, ld: int, t_dev_ptr: int):
    g = np.zeros(DE_MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(load().de_mlp_grad(m, ctypes.c_void_p(x_dev_ptr), ld, ctypes.c_void_p(t_dev_ptr), g.ctypes.data_as(_fp),
                              ctypes.byref(loss)), None)
    return g, loss.value


def de_mlp_train(m, x_dev_ptr: int, ld: int, t_dev_ptr: int, n: int, steps: int, lr: float = 1e-3):
    loss = ctypes.c_float()
    _check(load().de_mlp_train(m, ctypes.c_void_p(x_dev_ptr), ld, ctypes.c_void_p(t_dev_ptr), n, steps, lr,
                               ctypes.byref(loss)), None)
    return loss.value


def de_get_shape(h, run: int = 0):
    np_, d, nr = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().de_get_shape(h, run, ctypes.byref(np_), ctypes.byref(d), ctypes.byref(nr)), h)
    return np_.value, d.value, nr.value


def de_get_population(h, run: int = 0):
    np_, d, _ = de_get_shape(h, run)
    x = np.zeros((np_, d))
    f = np.zeros(np_)
    _check(load().de_get_population(h, run, _p(x), _p(f)), h)
    return x, f


def de_set_population(h, run: int, x, f=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    fa = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
    _check(load().de_set_population(h, run, _p(x), _p(fa)), h)


def de_set_generation(h, run: int, generation: int):
    _check(load().de_set_generation(h, run, generation), h)


def de_init_islands(cfg, nislands: int, interval: int, migrants: int, stream=None):
    """The island model: nislands copies of cfg (run_id + k) with ring
    migration every `interval` generations; returns the handle."""
    h = ctypes.c_void_p()
    _check(load().de_init_islands(ctypes.byref(cfg), nislands, interval, migrants, ctypes.c_void_p(stream or 0),
                                  ctypes.byref(h)), None)
    return h.value


def de_init_islands_ex(cfg, nislands: int, interval: int, migrants: int, migration: int, stream=None):
    """de_init_islands with a migration strategy (DE_MIGRATE_SYNC or
    DE_MIGRATE_ASYNC: migrants one interval late, through a mailbox)."""
    h = ctypes.c_void_p()
    _check(load().de_init_islands_ex(ctypes.byref(cfg), nislands, interval, migrants, migration,
                                     ctypes.c_void_p(stream or 0), ctypes.byref(h)), None)
    return h.value


def de_selftest_f32_rounding(x) -> int:
    """Mismatches between the library's FP64 -> FP32 rounding and the GPU's."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    return int(load().de_selftest_f32_rounding(_p(a), a.size))


def de_selftest_fp64_rate() -> float:
    """Measured FP64 fused multiply-add throughput of the current device (TFLOP/s)."""
    r = float(load().de_selftest_fp64_rate())
    if r <= 0:
        raise DEError(DE_ERR_CUDA, "FP64 rate self-test failed")
    return r


def de_get_adaptive(h, run: int = 0):
    """jDE parameters (F_i, CR_i) of the current population."""
    np_, _, _ = de_get_shape(h, run)
    F = np.empty(np_, dtype=np.float64)
    CR = np.empty(np_, dtype=np.float64)
    _check(load().de_get_adaptive(h, run, _p(F), _p(CR)), h)
    return F, CR


def de_set_adaptive(h, run: int, F=None, CR=None):
    np_, _, _ = de_get_shape(h, run)
    Fa = None if F is None else np.ascontiguousarray(F, dtype=np.float64).reshape(np_)
    Ca = None if CR is None else np.ascontiguousarray(CR, dtype=np.float64).reshape(np_)
    _check(load().de_set_adaptive(h, run, _p(Fa), _p(Ca)), h)


def de_get_best(h, run: int = 0):
    _, d, _ = de_get_shape(h, run)
    bf, bi = ctypes.c_double(), ctypes.c_int32()
    g, ev, sr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    bx = np.zeros(d)
    _check(load().de_get_best(h, run, ctypes.byref(bf), ctypes.byref(bi), _p(bx), ctypes.byref(g), ctypes.byref(ev),
                              ctypes.byref(sr)), h)
    return dict(best_f=bf.value, best_index=bi.value, best_x=bx, generations=g.value, evals=ev.value,
                stop_reason=sr.value)


def de_get_debug(h, run: int = 0):
    np_, d, _ = de_get_shape(h, run)
    nw = (d + 31) // 32
    out = dict(idx=np.zeros((np_, 3), np.int32), jrand=np.zeros(np_, np.int32), mask=np.zeros((np_, nw), np.uint32),
               trial=np.zeros((np_, d)), f_trial=np.zeros(np_), accept=np.zeros(np_, np.uint8),
               fp64_checked=np.zeros(np_, np.uint8), cand=np.zeros(np_, np.int32))
    dbg = de_debug(_p(out["idx"], _i32p), _p(out["jrand"], _i32p), _p(out["mask"], _u32p), _p(out["trial"]),
                   _p(out["f_trial"]), _p(out["accept"], _u8p), _p(out["fp64_checked"], _u8p),
                   _p(out["cand"], _i32p))
    _check(load().de_get_debug(h, run, ctypes.byref(dbg)), h)
    return out


def de_get_surrogate_stats(h):
    tr, sc, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    rho = ctypes.c_double()
    _check(load().de_get_surrogate_stats(h, ctypes.byref(tr), ctypes.byref(sc), ctypes.byref(rho), ctypes.byref(k)), h)
    return dict(trainings=tr.value, screened_generations=sc.value, last_rho=rho.value, k_now=k.value)


def de_get_stats(h, run: int = 0):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().de_get_stats(h, run, ctypes.byref(a), ctypes.byref(b)), h)
    return dict(fp64_reevals=a.value, trials=b.value)


def de_get_plan(h):
    p, c = ctypes.c_int32(), ctypes.c_int32()
    _check(load().de_get_plan(h, ctypes.byref(p), ctypes.byref(c)), h)
    return dict(kernel_path=p.value, cluster_size=c.value)


def de_save(h, path: str):
    _check(load().de_save(h, path.encode()), h)


def de_load(h, path: str):
    _check(load().de_load(h, path.encode()), h)


def de_destroy(h):
    _check(load().de_destroy(h))
