"""The FP64 cooperative persistent kernel (kernel path 3: every generation of
a single run in one launch, a grid barrier between generations) computes
exactly what the one-kernel-per-generation path computes, and follows the
CPU oracle; through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import capi, problems

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _cfgs():
    s = problems.suite(18, 10, seed=4)
    return [
        capi.make_config(64, 10, objective=0, shift=problems.shift(10, seed=1), seed=1, max_generations=10**6,
                         target_error=0.0),
        capi.make_config(250, 100, f=0.5, cr=0.3, objective=1, shift=problems.shift(100, seed=2),
                         rot=problems.rotation(100, seed=2), seed=2, max_generations=10**6, target_error=0.0),
        capi.make_config(100, 30, objective=3, shift=problems.shift(30, seed=3), rot=problems.rotation(30, seed=3),
                         seed=3, max_generations=10**6, target_error=0.0, strategy=capi.DE_RAND1EXP, jde=True),
        capi.make_config(48, 10, objective=18, shift=s["shift"], rot=s["rot"], perm=s["perm"], scale=s["scale"],
                         seed=4, max_generations=10**6, target_error=0.0, strategy=capi.DE_BEST1BIN),
        capi.make_config(16, 20, objective=4, shift=problems.ode_hidden(5), seed=5, max_generations=10**6,
                         target_error=0.0),
    ]


def _run(monkeypatch, persist, cfg, G):
    monkeypatch.setenv("DE_GB300_FP64_PERSIST", "1" if persist else "0")
    h = capi.de_init(cfg)
    try:
        plan = capi.de_get_plan(h)["kernel_path"]
        capi.de_step(h, G)
        x, f = capi.de_get_population(h)
        b = capi.de_get_best(h)
        ad = capi.de_get_adaptive(h) if cfg.jde else None
    finally:
        capi.de_destroy(h)
    assert plan == (3 if persist else 0)
    return x, f, b, ad


@pytest.mark.parametrize("k", range(5))
def test_persistent_fp64_equals_the_per_generation_kernel(k, monkeypatch):
    _need_gpu()
    G = 120
    xa, fa, ba, ada = _run(monkeypatch, True, _cfgs()[k], G)
    xb, fb, bb, adb = _run(monkeypatch, False, _cfgs()[k], G)
    assert np.array_equal(xa, xb) and np.array_equal(fa, fb)
    for key in ("generations", "evals", "best_index", "best_f", "stop_reason"):
        assert ba[key] == bb[key], key
    assert ba["generations"] == G
    if ada is not None:
        assert np.array_equal(ada[0], adb[0]) and np.array_equal(ada[1], adb[1])


def test_persistent_fp64_runs_the_small_sphere_like_the_oracle(monkeypatch):
    _need_gpu()
    monkeypatch.setenv("DE_GB300_FP64_PERSIST", "1")
    d = 10
    o = problems.shift(d, seed=1)
    Xo, fo, go, evo, _ = oracle.run(64, d, 0.5, 0.9, -100, 100, 0, o, None, seed=1, max_generations=1000,
                                    target_error=1e-8)
    h = capi.de_init(capi.make_config(64, d, objective=0, shift=o, seed=1, max_generations=1000, target_error=1e-8))
    try:
        assert capi.de_get_plan(h)["kernel_path"] == 3
        res = capi.de_run(h)[0]
        x, f = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    assert res["generations"] == go and res["evals"] == evo and res["stop_reason"] == capi.DE_STOP_TARGET
    assert np.array_equal(x, Xo)
    assert np.allclose(f, fo, rtol=1e-12, atol=0)


def test_persistent_fp64_one_generation_matches_oracle(monkeypatch):
    _need_gpu()
    monkeypatch.setenv("DE_GB300_FP64_PERSIST", "1")
    np_, d, obj = 300, 37, 2
    o, M = problems.shift(d, seed=8), problems.rotation(d, seed=8)
    X = problems.population(np_, d, seed=8)
    fX, _ = oracle.evaluate(obj, X, o, M)
    h = capi.de_init(capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=9, max_generations=100,
                                      target_error=0.0, debug_capture=True))
    try:
        assert capi.de_get_plan(h)["kernel_path"] == 3
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, 4)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        best = capi.de_get_best(h)
    finally:
        capi.de_destroy(h)
    r = oracle.step(X, fX, 0.5, 0.9, -100, 100, obj, o, M, seed=9, generation=5)
    assert np.array_equal(g["idx"], r["idx"]) and np.array_equal(g["mask"], r["mask"])
    assert np.array_equal(g["trial"], r["trial"])
    tol = 1e-12 * (np.abs(r["f_trial"]) + r["sabs_trial"])
    assert np.all(np.abs(g["f_trial"] - r["f_trial"]) <= tol)
    band = np.abs(r["f_trial"] - fX) <= tol
    assert np.array_equal(g["accept"][~band], r["accept"][~band])
    assert best["generations"] == 5 and best["evals"] == np_ * 6


def _batch_cfgs():
    """Uneven runs that stop at different generations: by the target, by the
    evaluation budget and by the generation limit."""
    s17 = problems.suite(17, 20, seed=6)
    return [
        capi.make_config(32, 5, objective=0, shift=problems.shift(5, seed=1), seed=1, max_generations=400,
                         target_error=1e-6),
        capi.make_config(64, 10, objective=0, shift=problems.shift(10, seed=2), seed=2, run_id=1,
                         max_generations=5000, target_error=1e-8),
        capi.make_config(40, 17, objective=2, shift=problems.shift(17, seed=3), rot=problems.rotation(17, seed=3),
                         seed=3, max_evals=40 * 90, max_generations=10**6, target_error=0.0),
        capi.make_config(24, 20, objective=17, shift=s17["shift"], rot=s17["rot"], perm=s17["perm"],
                         scale=s17["scale"], seed=6, max_generations=150, target_error=0.0, jde=True),
        capi.make_config(90, 33, objective=1, shift=problems.shift(33, seed=7), seed=7, max_generations=260,
                         target_error=0.0, strategy=capi.DE_BEST1BIN),
    ]


def _run_batch(monkeypatch, persist, steps):
    monkeypatch.setenv("DE_GB300_FP64_PERSIST", "1" if persist else "0")
    cfgs = _batch_cfgs()
    h = capi.de_init_batch(cfgs)
    out = []
    try:
        plan = capi.de_get_plan(h)["kernel_path"]
        for n in steps:
            if n < 0:
                capi.de_reset(h, -n - 1)
            else:
                capi.de_step(h, n)
        for r in range(len(cfgs)):
            x, f = capi.de_get_population(h, r)
            out.append((x, f, capi.de_get_best(h, r)))
    finally:
        capi.de_destroy(h)
    assert plan == (3 if persist else 0)
    return out


@pytest.mark.parametrize("steps", [[5000], [37, 1, 200, 4000], [100, -2, 60, -5, 3000]])
def test_persistent_fp64_batch_equals_the_per_generation_kernel(steps, monkeypatch):
    """Runs stop at different generations (a stopped run's tiles keep meeting
    the grid barrier until the last run stops); resets of single runs."""
    _need_gpu()
    a = _run_batch(monkeypatch, True, steps)
    b = _run_batch(monkeypatch, False, steps)
    for r, ((xa, fa, ba), (xb, fb, bb)) in enumerate(zip(a, b)):
        assert np.array_equal(xa, xb) and np.array_equal(fa, fb), r
        for key in ("generations", "evals", "best_index", "best_f", "stop_reason"):
            assert ba[key] == bb[key], (r, key)
    stops = [x[2]["stop_reason"] for x in a]
    if steps == [5000]:
        assert stops[0] == capi.DE_STOP_TARGET and stops[2] == capi.DE_STOP_EVALS
        assert stops[3] == capi.DE_STOP_GENERATIONS and stops[4] == capi.DE_STOP_GENERATIONS


def test_persistent_fp64_batch_runs_like_the_oracle(monkeypatch):
    _need_gpu()
    monkeypatch.setenv("DE_GB300_FP64_PERSIST", "1")
    cfgs = _batch_cfgs()[:3]
    h = capi.de_init_batch(cfgs)
    try:
        assert capi.de_get_plan(h)["kernel_path"] == 3
        capi.de_step(h, 5000)
        got = [(capi.de_get_population(h, r), capi.de_get_best(h, r)) for r in range(3)]
    finally:
        capi.de_destroy(h)
    args = [(32, 5, 0, problems.shift(5, seed=1), None, 1, 0, 400, 0, 1e-6),
            (64, 10, 0, problems.shift(10, seed=2), None, 2, 1, 5000, 0, 1e-8),
            (40, 17, 2, problems.shift(17, seed=3), problems.rotation(17, seed=3), 3, 0, 10**6, 40 * 90, 0.0)]
    for (np_, d, obj, o, M, seed, rid, mg, me, te), ((x, f), b) in zip(args, got):
        Xo, fo, go, evo, _ = oracle.run(np_, d, 0.5, 0.9, -100, 100, obj, o, M, seed=seed, run_id=rid,
                                        max_generations=mg, max_evals=me, target_error=te)
        assert b["generations"] == go and b["evals"] == evo
        assert np.array_equal(x, Xo)
        assert np.allclose(f, fo, rtol=1e-12, atol=0)


def _small_cfgs():
    """Runs of at most 8 tiles: the cooperative loop can run as one
    thread-block cluster (rows per tile 1 without the autotuner)."""
    s19 = problems.suite(19, 12, seed=9)
    return [
        capi.make_config(8, 10, objective=0, shift=problems.shift(10, seed=1), seed=1, max_generations=10**6,
                         target_error=0.0),
        capi.make_config(7, 37, objective=1, shift=problems.shift(37, seed=2), rot=problems.rotation(37, seed=2),
                         seed=2, max_generations=10**6, target_error=0.0, jde=True, strategy=capi.DE_RAND1EXP),
        capi.make_config(5, 12, objective=19, shift=s19["shift"], rot=s19["rot"], seed=9, max_generations=10**6,
                         target_error=0.0, strategy=capi.DE_BEST1BIN),
    ]


@pytest.mark.parametrize("k", range(3))
def test_one_cluster_fp64_loop_equals_the_per_generation_kernel(k, monkeypatch):
    """The cooperative FP64 loop launched as one cluster (cluster barrier
    between generations) gives the populations, records and jDE parameters of
    the one-kernel-per-generation path."""
    _need_gpu()
    monkeypatch.setenv("DE_GB300_AUTOTUNE", "0")
    out = []
    for mode in ("2", "0"):
        monkeypatch.setenv("DE_GB300_FP64_PERSIST", mode)
        cfg = _small_cfgs()[k]
        h = capi.de_init(cfg)
        try:
            plan = capi.de_get_plan(h)
            capi.de_step(h, 150)
            x, f = capi.de_get_population(h)
            out.append((plan, x, f, capi.de_get_best(h), capi.de_get_adaptive(h) if cfg.jde else None))
        finally:
            capi.de_destroy(h)
    (pa, xa, fa, ba, ada), (pb, xb, fb, bb, adb) = out
    assert pa == {"kernel_path": 3, "cluster_size": _small_cfgs()[k].np} and pb["kernel_path"] == 0
    assert np.array_equal(xa, xb) and np.array_equal(fa, fb)
    for key in ("generations", "evals", "best_index", "best_f", "stop_reason"):
        assert ba[key] == bb[key], key
    assert ba["generations"] == 150
    if ada is not None:
        assert np.array_equal(ada[0], adb[0]) and np.array_equal(ada[1], adb[1])


def test_one_cluster_fp64_run_stops_like_the_oracle(monkeypatch):
    """A run to 1e-8 as one cluster stops at the oracle's generation with its
    evaluation count, and its population equals the per-generation path's
    (near the optimum the GPU and the oracle may settle FP64 near-ties
    differently, so the oracle's population is not compared)."""
    _need_gpu()
    monkeypatch.setenv("DE_GB300_AUTOTUNE", "0")
    d = 6
    o = problems.shift(d, seed=3)
    Xo, fo, go, evo, _ = oracle.run(8, d, 0.5, 0.9, -100, 100, 0, o, None, seed=3, max_generations=3000,
                                    target_error=1e-8)
    out = []
    for mode in ("2", "0"):
        monkeypatch.setenv("DE_GB300_FP64_PERSIST", mode)
        h = capi.de_init(capi.make_config(8, d, objective=0, shift=o, seed=3, max_generations=3000,
                                          target_error=1e-8))
        try:
            assert capi.de_get_plan(h)["cluster_size"] == (8 if mode == "2" else 0)
            res = capi.de_run(h)[0]
            out.append((res, capi.de_get_population(h)))
        finally:
            capi.de_destroy(h)
    (ra, (xa, fa)), (rb, (xb, fb)) = out
    assert ra["generations"] == rb["generations"] == go and ra["evals"] == rb["evals"] == evo
    assert ra["stop_reason"] == rb["stop_reason"]
    assert np.array_equal(xa, xb) and np.array_equal(fa, fb)
