"""FP64 CPU oracle of DE/rand/1/bin (arXiv 2405.16551, Sec. 2 and Sec. 7.3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never imports it, never links it, and shares no
code with it; it exists to check the CUDA path.

The arithmetic lives in plain C (``de_oracle.c``, ``de_oracle_ode.c``,
``de_oracle_mlp.c``, ``de_oracle_suite.c``, ``de_oracle_islands.c``), compiled with gcc on first use (or by ``build()``) and
called through ctypes.  This module only marshals numpy arrays.

Parity pins for every function are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["de_oracle.c", "de_oracle_ode.c", "de_oracle_mlp.c", "de_oracle_suite.c", "de_oracle_islands.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "libde_oracle.so")
_lib = None
_lock = threading.Lock()

SPHERE, RASTRIGIN, ROSENBROCK, ACKLEY = 0, 1, 2, 3
PURPOSE_INIT, PURPOSE_STEP = 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``_build/libde_oracle.so``."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.or_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        lib.or_draw.restype = ctypes.c_uint32
        lib.or_map.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        lib.or_map.restype = ctypes.c_uint32
        lib.or_u53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        lib.or_u53.restype = ctypes.c_double
        lib.or_cr_threshold.argtypes = [ctypes.c_double]
        lib.or_cr_threshold.restype = ctypes.c_uint64
        lib.or_mutant_indices.argtypes = [ctypes.c_uint32] * 5 + [_u32p]
        lib.or_objective.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp]
        lib.or_objective.restype = ctypes.c_double
        lib.or_eval.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp,
                                ctypes.c_int64, ctypes.c_int, _dp, _dp, ctypes.c_int]
        lib.or_eval_p.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _i32p, _dp,
                                  ctypes.c_int64, ctypes.c_int, _dp, _dp, ctypes.c_int]
        lib.or_objective_p.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _i32p, _dp, _dp]
        lib.or_objective_p.restype = ctypes.c_double
        lib.or_basic.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        lib.or_basic.restype = ctypes.c_double
        lib.or_domain_scale.argtypes = [ctypes.c_int]
        lib.or_domain_scale.restype = ctypes.c_double
        lib.or_hybrid_segments.argtypes = [ctypes.c_int, ctypes.c_int, _i32p]
        lib.or_hybrid_segments.restype = ctypes.c_int
        lib.or_suite_components.argtypes = [ctypes.c_int]
        lib.or_suite_components.restype = ctypes.c_int
        lib.or_island_ranked.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _i32p]
        lib.or_run_islands.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, _dp, _dp, _i32p, ctypes.c_double, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_double, _dp, _dp, _dp, _dp, _i64p, ctypes.c_int, ctypes.c_int]
        lib.or_run_islands.restype = ctypes.c_int64
        lib.or_init_population.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_uint64, ctypes.c_uint32, _dp]
        lib.or_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                _dp, _dp, _dp, _dp, _i32p, _i32p, _u32p, _dp, _dp, _dp, _u8p, ctypes.c_int]
        lib.or_step_cand.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                     ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _i32p,
                                     _dp, _dp, _dp, _dp, _i32p, _i32p, _u32p, _dp, _dp, _dp, _u8p, ctypes.c_int]
        lib.or_step_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, _i32p, ctypes.c_double,
                                   ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _i32p, ctypes.c_int, ctypes.c_int,
                                   _dp, _dp, _dp, _dp,
                                   _dp, _dp, _dp, _dp, _i32p, _i32p, _u32p, _dp, _dp, _dp, _u8p, ctypes.c_int]
        lib.or_run_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, _i32p, ctypes.c_double,
                                  ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_double, _dp, _dp, _dp, _dp, _i64p, _dp, ctypes.c_int]
        lib.or_run_ex.restype = ctypes.c_int64
        lib.or_best.argtypes = [ctypes.c_int, _dp]
        lib.or_best.restype = ctypes.c_int
        lib.or_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_double,
                               ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_double, _dp, _dp, _i64p, _dp, ctypes.c_int]
        lib.or_run.restype = ctypes.c_int64
        _bind_extra(lib)
        _lib = lib
        return lib


def _bind_extra(lib):
    """Bindings of the ODE and MLP parts (present once their sources exist)."""
    if hasattr(lib, "or_ode_objective"):
        lib.or_ode_objective.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double]
        lib.or_ode_objective.restype = ctypes.c_double
        lib.or_ode_objective_s.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double, _dp]
        lib.or_ode_objective_s.restype = ctypes.c_double
        lib.or_ode_trajectory.argtypes = [_dp, ctypes.c_int, ctypes.c_double, _dp]
        lib.or_ode_integrate.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double, _dp]
        lib.or_ode_params.argtypes = [_dp, _dp, _dp]
    if hasattr(lib, "or_mlp_forward"):
        lib.or_mlp_forward.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int] + [_dp] * 8
        lib.or_mlp_loss_grad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int] + [_dp] * 14
        lib.or_mlp_loss_grad.restype = ctypes.c_double
        lib.or_adam.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double]


def _p(a, t=_dp):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


# ----------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def draw(seed, purpose, run_id, cand, generation, individual, d):
    return int(_load().or_draw(seed, purpose, run_id, cand, generation, individual, d))


def map_index(u, n):
    return int(_load().or_map(u, n))


def u53(a, b):
    return float(_load().or_u53(a, b))


def cr_threshold(cr):
    return int(_load().or_cr_threshold(cr))


def mutant_indices(w0, w1, w2, i, np_):
    r = np.zeros(3, dtype=np.uint32)
    _load().or_mutant_indices(w0, w1, w2, i, np_, _p(r, _u32p))
    return tuple(int(v) for v in r)


# ----------------------------------------------------------------------------- objectives
def objective(obj, x, o=None, M=None, scale=1.0, perm=None):
    """f(x) and the magnitude sum of its terms for one point."""
    x = _f64(x)
    d = x.shape[0]
    o, M = _f64(o), _f64(M)
    sabs = ctypes.c_double(0.0)
    f = _load().or_objective_p(obj, d, _p(o), _p(M), scale, _p(_i32(perm), _i32p), _p(x), ctypes.byref(sabs))
    return f, sabs.value


# ----------------------------------------------------------------------------- benchmark suite (Table 2)
ZAKHAROV, SCHWEFEL, BENT_CIGAR, HGBAT, SCHAFFER_F6, KATSUURA, HAPPYCAT = 5, 6, 7, 8, 9, 10, 11
GRIEWANK_ROSENBROCK, ELLIPTIC, GRIEWANK = 12, 13, 14
HYBRID1, HYBRID2, HYBRID3, COMPOSITION1, COMPOSITION2, COMPOSITION3 = 15, 16, 17, 18, 19, 20


def basic(fn, z, e=None):
    """(g(z), tolerance scale) of basic function fn on the vector z."""
    z = _f64(np.atleast_1d(z))
    s = ctypes.c_double()
    f = _load().or_basic(fn, z.shape[0], _p(z), _p(_f64(e)), ctypes.byref(s))
    return f, s.value


def domain_scale(fn):
    return float(_load().or_domain_scale(fn))


def hybrid_segments(obj, d):
    """Start of every part of a hybrid function's split of d coordinates
    (m + 1 entries), or None when some part would be empty."""
    st = np.zeros(6, dtype=np.int32)
    m = _load().or_hybrid_segments(obj, d, _p(st, _i32p))
    return None if m == 0 else st[: m + 1].copy()


def suite_components(obj):
    return int(_load().or_suite_components(obj))


# ----------------------------------------------------------------------------- ODE objective
ODE = 4
ODE_STEPS, ODE_DT, ODE_N = 2000, 1e-3, 10


def ode_params(x):
    """(k, c) of the oscillator chain from a parameter vector of length 20."""
    x = _f64(x)
    k = np.zeros(ODE_N)
    c = np.zeros(ODE_N)
    _load().or_ode_params(_p(x), _p(k), _p(c))
    return k, c


def ode_integrate(k, c, steps=ODE_STEPS, dt=ODE_DT):
    """Positions after every RK4 step (steps x 10) for raw parameters k, c."""
    out = np.zeros((steps, ODE_N))
    _load().or_ode_integrate(_p(_f64(k)), _p(_f64(c)), steps, dt, _p(out))
    return out


def ode_trajectory(x, steps=ODE_STEPS, dt=ODE_DT):
    out = np.zeros((steps, ODE_N))
    _load().or_ode_trajectory(_p(_f64(x)), steps, dt, _p(out))
    return out


def ode_objective(x, x_hat, steps=ODE_STEPS, dt=ODE_DT):
    """(f, tolerance scale S) of the ODE fitting objective."""
    s = ctypes.c_double()
    f = _load().or_ode_objective_s(_p(_f64(x)), _p(_f64(x_hat)), steps, dt, ctypes.byref(s))
    return f, s.value


# ----------------------------------------------------------------------------- surrogate MLP
MLP_KEYS = ("W1", "b1", "W2", "b2", "w3", "b3")


def mlp_forward(params, X):
    """y for every row of X; params = dict of W1 (nh x nin), b1, W2 (nh x nh), b2, w3, b3."""
    X = _f64(np.atleast_2d(X))
    B, nin = X.shape
    p = {k: _f64(np.atleast_1d(params[k])) for k in MLP_KEYS}
    nh = p["b1"].shape[0]
    y = np.zeros(B)
    _load().or_mlp_forward(B, nin, nh, _p(X), _p(p["W1"]), _p(p["b1"]), _p(p["W2"]), _p(p["b2"]), _p(p["w3"]),
                           _p(p["b3"]), _p(y))
    return y


def mlp_loss_grad(params, X, t):
    """(loss, grads) with grads keyed like params."""
    X = _f64(np.atleast_2d(X))
    B, nin = X.shape
    p = {k: _f64(np.atleast_1d(params[k])) for k in MLP_KEYS}
    g = {k: np.zeros_like(p[k]) for k in MLP_KEYS}
    loss = _load().or_mlp_loss_grad(B, nin, p["b1"].shape[0], _p(X), _p(_f64(t)), *[_p(p[k]) for k in MLP_KEYS],
                                    *[_p(g[k]) for k in MLP_KEYS])
    return loss, g


def adam(w, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place on float64 arrays w, m, v with gradient g."""
    for a in (w, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _load().or_adam(w.size, _p(w), _p(_f64(g)), _p(m), _p(v), step, lr, beta1, beta2, eps)


def evaluate(obj, X, o=None, M=None, scale=1.0, threads=1, perm=None):
    """f and magnitude sums for every row of X."""
    X = _f64(X)
    n, d = X.shape
    f = np.zeros(n)
    sabs = np.zeros(n)
    _load().or_eval_p(obj, d, _p(_f64(o)), _p(_f64(M)), scale, _p(_i32(perm), _i32p), _p(X), d, n, _p(f), _p(sabs),
                      threads)
    return f, sabs


# ----------------------------------------------------------------------------- DE
def init_population(np_, d, lo, hi, seed, run_id=0):
    X = np.zeros((np_, d))
    _load().or_init_population(np_, d, lo, hi, seed, run_id, _p(X))
    return X


STRATEGIES = {"rand1bin": 0, "best1bin": 1, "rand1exp": 2}


def step(X, fX, F, CR, lo, hi, obj, o, M, seed, generation, run_id=0, scale=1.0, threads=1, cand=None,
         strategy=0, jde=False, jF=None, jCR=None, perm=None):
    """One synchronous generation; returns a dict with the next population and
    every intermediate (indices, j_rand (the crossover start for exp),
    crossover mask, trials, f_trial, magnitude sums, accept flags).  cand:
    per-target candidate stream (None: stream 0, plain DE).  strategy: 0
    rand/1/bin, 1 best/1/bin, 2 rand/1/exp.  jde: per-individual F and CR
    (jF, jCR of generation g - 1, default all F / CR); the dict then carries
    F_next and CR_next."""
    X = _f64(X)
    fX = _f64(fX)
    np_, d = X.shape
    nw = (d + 31) // 32
    out = dict(
        X_next=np.zeros_like(X), f_next=np.zeros(np_), idx=np.zeros((np_, 3), dtype=np.int32),
        jrand=np.zeros(np_, dtype=np.int32), mask=np.zeros((np_, nw), dtype=np.uint32),
        trial=np.zeros_like(X), f_trial=np.zeros(np_), sabs_trial=np.zeros(np_),
        accept=np.zeros(np_, dtype=np.uint8))
    cnd = None if cand is None else np.ascontiguousarray(cand, dtype=np.int32)
    jFa = jCRa = None
    if jde:
        jFa = np.full(np_, F) if jF is None else _f64(jF)
        jCRa = np.full(np_, CR) if jCR is None else _f64(jCR)
        out["F_next"] = np.zeros(np_)
        out["CR_next"] = np.zeros(np_)
    _load().or_step_ex(np_, d, F, CR, lo, hi, obj, _p(_f64(o)), _p(_f64(M)), _p(_i32(perm), _i32p), scale, seed,
                    run_id, generation,
                    _p(cnd, _i32p), int(strategy), 1 if jde else 0, _p(jFa), _p(jCRa),
                    _p(out.get("F_next")), _p(out.get("CR_next")), _p(X), _p(fX), _p(out["X_next"]), _p(out["f_next"]), _p(out["idx"], _i32p),
                    _p(out["jrand"], _i32p), _p(out["mask"], _u32p), _p(out["trial"]), _p(out["f_trial"]),
                    _p(out["sabs_trial"]), _p(out["accept"], _u8p), threads)
    return out


def best(f):
    f = _f64(f)
    return int(_load().or_best(f.shape[0], _p(f)))


def run(np_, d, F, CR, lo, hi, obj, o, M, seed, max_generations, max_evals=0, target_error=1e-8,
        run_id=0, scale=1.0, threads=1, trace=False, strategy=0, jde=False, return_adaptive=False, perm=None):
    """A whole run; returns (X, f, generations, evals, best_trace or None),
    and (F_i, CR_i) after them when return_adaptive (jde)."""
    X = np.zeros((np_, d))
    f = np.zeros(np_)
    jF = np.zeros(np_)
    jCR = np.zeros(np_)
    ev = ctypes.c_int64(0)
    tr = np.full(max_generations + 1, np.nan) if trace else None
    g = _load().or_run_ex(np_, d, F, CR, lo, hi, obj, _p(_f64(o)), _p(_f64(M)), _p(_i32(perm), _i32p), scale, seed,
                          run_id, int(strategy),
                          1 if jde else 0, max_generations, max_evals, target_error, _p(X), _p(f), _p(jF), _p(jCR),
                          ctypes.byref(ev), _p(tr), threads)
    res = (X, f, int(g), int(ev.value), (tr[: g + 1] if trace else None))
    return res + (jF, jCR) if return_adaptive else res


# ----------------------------------------------------------------------------- island model
def island_ranked(f, n, worst=False):
    """The n best (or worst) indices of f in the island model's order."""
    f = _f64(f)
    out = np.zeros(n, dtype=np.int32)
    _load().or_island_ranked(f.shape[0], _p(f), n, 1 if worst else 0, _p(out, _i32p))
    return out


def run_islands(m, interval, nmig, np_, d, F, CR, lo, hi, obj, o, M, seed, max_generations, max_evals=0,
                target_error=1e-8, run_id=0, scale=1.0, perm=None, strategy=0, jde=False, threads=1,
                asynchronous=False):
    """The island model: returns (X [m, np, d], f [m, np], generations,
    evaluations of one island, F_i [m, np], CR_i [m, np]).  asynchronous:
    migrants arrive one migration interval late (posted at the previous
    migration point)."""
    X = np.zeros((m, np_, d))
    f = np.zeros((m, np_))
    jF = np.zeros((m, np_))
    jCR = np.zeros((m, np_))
    ev = ctypes.c_int64(0)
    g = _load().or_run_islands(m, interval, nmig, np_, d, F, CR, lo, hi, obj, _p(_f64(o)), _p(_f64(M)),
                               _p(_i32(perm), _i32p), scale, seed, run_id, int(strategy), 1 if jde else 0,
                               max_generations, max_evals, target_error, _p(X), _p(f), _p(jF), _p(jCR),
                               ctypes.byref(ev), threads, 1 if asynchronous else 0)
    return X, f, int(g), int(ev.value), jF, jCR
