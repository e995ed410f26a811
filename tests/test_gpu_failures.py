"""Failure detection without a GPU fault, through the C ABI.

  * a bounded device wait that runs out: the cooperative FP64 kernel's grid
    barrier, with one CTA leaving out its first arrival (the library's test
    switch DE_GB300_TEST_GRID_TIMEOUT) and a short poll limit; the call
    returns DE_ERR_TIMEOUT and the device stays usable;
  * non-finite fitness: a NaN trial is never selected (Sec. 2 selection, as
    the oracle takes it), on every precision; a run whose whole population
    has NaN fitness reports DE_ERR_NONFINITE;
  * a device allocation that fails: DE_ERR_OOM, and nothing stays allocated;
  * checkpoints written for another problem are refused before anything is
    copied to the device.
"""
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


# ----------------------------------------------------------------------------- bounded waits
def test_grid_barrier_timeout_is_reported_and_the_device_stays_usable(monkeypatch):
    _need_gpu()
    np_, d, obj = 1024, 100, 1
    o, M = problems.shift(d, seed=21), problems.rotation(d, seed=21)
    monkeypatch.setenv("DE_GB300_FP64_PERSIST", "1")
    monkeypatch.setenv("DE_GB300_AUTOTUNE", "0")
    monkeypatch.setenv("DE_GB300_TEST_GRID_TIMEOUT", "1")
    cfg = capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=3, max_generations=50, target_error=0.0)
    h = capi.de_init(cfg)
    try:
        assert capi.de_get_plan(h)["kernel_path"] == 3  # the cooperative FP64 kernel
        with pytest.raises(capi.DEError) as ei:
            capi.de_run(h)
        assert ei.value.status == capi.DE_ERR_TIMEOUT
        # the barrier gave up in the first generation: no generation completed
        assert capi.de_get_best(h)["generations"] == 0
    finally:
        capi.de_destroy(h)
    # same device, new handle without the test switch: one generation equals the oracle's
    monkeypatch.delenv("DE_GB300_TEST_GRID_TIMEOUT")
    X = problems.population(np_, d, seed=22)
    fX, _ = oracle.evaluate(obj, X, o, M)
    h = capi.de_init(capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=3, max_generations=50,
                                      target_error=0.0, debug_capture=True))
    try:
        assert capi.de_get_plan(h)["kernel_path"] == 3
        capi.de_set_population(h, 0, X, fX)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        r = capi.de_run(h)[0]
    finally:
        capi.de_destroy(h)
    ref = oracle.step(X, fX, 0.5, 0.9, -100, 100, obj, o, M, seed=3, generation=1)
    assert np.array_equal(g["trial"], ref["trial"])
    tol = 1e-12 * (np.abs(ref["f_trial"]) + ref["sabs_trial"])
    assert np.all(np.abs(g["f_trial"] - ref["f_trial"]) <= tol)
    assert r["generations"] == 50 and r["stop_reason"] == capi.DE_STOP_GENERATIONS


@pytest.mark.parametrize("mode,path", [("cta", 4), ("cluster", 2)])
def test_split_persistent_grid_barrier_timeout_is_reported(mode, path, monkeypatch):
    """The split persistent kernels (the CTA-local one of the NP = 1024,
    D = 100 configuration, and the cluster form): CTA 0 leaves out its first
    grid-barrier arrival, every CTA's bounded wait gives up, the run reports
    DE_ERR_TIMEOUT with no generation completed, and the device stays usable."""
    _need_gpu()
    np_, d, obj = 1024, 100, 1
    o, M = problems.shift(d, seed=23), problems.rotation(d, seed=23)
    monkeypatch.setenv("DE_GB300_PERSIST_MODE", mode)
    monkeypatch.setenv("DE_GB300_AUTOTUNE", "0")
    monkeypatch.setenv("DE_GB300_TEST_GRID_TIMEOUT", "1")
    cfg = capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=4, precision=capi.DE_PREC_BF16X3,
                           max_generations=50, target_error=0.0)
    h = capi.de_init(cfg)
    try:
        assert capi.de_get_plan(h)["kernel_path"] == path
        with pytest.raises(capi.DEError) as ei:
            capi.de_run(h)
        assert ei.value.status == capi.DE_ERR_TIMEOUT
        assert capi.de_get_best(h)["generations"] == 0
    finally:
        capi.de_destroy(h)
    monkeypatch.delenv("DE_GB300_TEST_GRID_TIMEOUT")
    h = capi.de_init(cfg)
    try:
        assert capi.de_get_plan(h)["kernel_path"] == path
        r = capi.de_run(h)[0]
    finally:
        capi.de_destroy(h)
    assert r["generations"] == 50 and r["stop_reason"] == capi.DE_STOP_GENERATIONS


def test_batch_arrival_counter_timeout_is_reported(monkeypatch):
    """The persistent batch kernel: CTA 0 leaves out the arrival of its first
    item's first generation, the CTAs waiting for that run give up, the batch
    reports DE_ERR_TIMEOUT, and a new handle on the same device runs."""
    _need_gpu()
    shapes = [(150, 30, 1), (200, 20, 0), (90, 10, 3), (300, 50, 2)]
    cfgs = [capi.make_config(n, dd, objective=ob, shift=problems.shift(dd, seed=5, run_id=r),
                             rot=problems.rotation(dd, seed=5, run_id=r), seed=5, run_id=r,
                             precision=capi.DE_PREC_BF16X3, max_generations=40, target_error=0.0)
            for r, (n, dd, ob) in enumerate(shapes)]
    monkeypatch.setenv("DE_GB300_PERSIST_BATCH", "1")
    monkeypatch.setenv("DE_GB300_TEST_GRID_TIMEOUT", "1")
    h = capi.de_init_batch(cfgs)
    try:
        assert capi.de_get_plan(h)["kernel_path"] == 5
        with pytest.raises(capi.DEError) as ei:
            capi.de_run(h, len(cfgs))
        assert ei.value.status == capi.DE_ERR_TIMEOUT
    finally:
        capi.de_destroy(h)
    monkeypatch.delenv("DE_GB300_TEST_GRID_TIMEOUT")
    h = capi.de_init_batch(cfgs)
    try:
        assert capi.de_get_plan(h)["kernel_path"] == 5
        res = capi.de_run(h, len(cfgs))
    finally:
        capi.de_destroy(h)
    assert all(r["generations"] == 40 for r in res)


# ----------------------------------------------------------------------------- NaN fitness
def _nan_problem(np_, d, seed, values):
    """Unrotated Rastrigin with o = 0 and scale 1e308 on a population whose
    coordinates are drawn from `values` (0 or magnitude >= 50): a trial
    coordinate is then 0 or at least 50 in magnitude (mutation with F = 0.5 and
    the midpoint repair keep it so), y = x * 1e308 is 0 or +-inf, and f is 0
    when every coordinate is 0, else NaN (cos(2 pi inf) is NaN) on both sides."""
    rng = np.random.default_rng(seed)
    X = rng.choice(values, size=(np_, d)).astype(np.float64)
    return X, np.zeros(d)


@pytest.mark.parametrize("prec", [capi.DE_PREC_FP64, capi.DE_PREC_BF16X3, capi.DE_PREC_TF32X3])
def test_nan_trials_are_never_selected(prec):
    _need_gpu()
    np_, d, scale, seed, gen = 64, 2, 1e308, 4, 5
    X, o = _nan_problem(np_, d, 30, [0.0, 100.0, -100.0])
    fX, _ = oracle.evaluate(1, X, o, None, scale=scale)
    assert np.isnan(fX).any() and (~np.isnan(fX)).any()
    cfg = capi.make_config(np_, d, objective=1, scale=scale, shift=o, seed=seed, precision=prec, max_generations=100,
                           target_error=0.0, debug_capture=True)
    h = capi.de_init(cfg)
    try:
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, gen - 1)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        x1, f1 = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    ref = oracle.step(X, fX, 0.5, 0.9, -100, 100, 1, o, None, seed=seed, generation=gen, scale=scale)
    assert np.isnan(ref["f_trial"]).any() and (~np.isnan(ref["f_trial"])).any()
    assert np.array_equal(g["trial"], ref["trial"])
    assert np.array_equal(g["accept"], ref["accept"])
    acc = g["accept"].astype(bool)
    assert not np.isnan(g["f_trial"][acc]).any()  # no NaN trial replaced its target
    assert np.array_equal(x1, ref["X_next"]) and np.array_equal(np.isnan(f1), np.isnan(ref["f_next"]))


def test_all_nan_fitness_reports_nonfinite():
    _need_gpu()
    np_, d, scale, seed, G = 32, 8, 1e308, 5, 3
    X, o = _nan_problem(np_, d, 31, [100.0, -100.0])
    fX = np.full(np_, np.nan)
    # the oracle keeps every fitness NaN over these generations (no trial is all zero)
    Xo, fo = X, fX
    for g in range(1, G + 1):
        ref = oracle.step(Xo, fo, 0.5, 0.5, -100, 100, 1, o, None, seed=seed, generation=g, scale=scale)
        assert not ref["accept"].any()
        Xo, fo = ref["X_next"], ref["f_next"]
    assert np.isnan(fo).all()
    h = capi.de_init(capi.make_config(np_, d, cr=0.5, objective=1, scale=scale, shift=o, seed=seed,
                                      max_generations=G, target_error=0.0))
    try:
        capi.de_set_population(h, 0, X, fX)
        with pytest.raises(capi.DEError) as ei:
            capi.de_run(h)
        assert ei.value.status == capi.DE_ERR_NONFINITE
        x1, f1 = capi.de_get_population(h)
        assert np.array_equal(x1, X) and np.isnan(f1).all()  # nothing was ever accepted
    finally:
        capi.de_destroy(h)


# ----------------------------------------------------------------------------- allocation failure
def test_device_allocation_failure_returns_oom_and_frees_everything():
    torch = _need_gpu()
    # warm-up: the CUDA context and the library's one-time state exist before measuring
    capi.de_destroy(capi.de_init(capi.make_config(16, 4, max_generations=1)))
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    # five runs of the largest accepted shape need about 343 GB of population
    # buffers alone, more than the device holds
    big = [capi.make_config(1 << 20, 4096, run_id=r, max_generations=1) for r in range(5)]
    assert 5 * 2 * (1 << 20) * 4096 * 8 > total
    with pytest.raises(capi.DEError) as ei:
        capi.de_init_batch(big)
    assert ei.value.status == capi.DE_ERR_OOM
    torch.cuda.synchronize()
    # nothing of the failed set-up stays allocated (free memory may only have
    # grown, by a deferred release of an earlier test's handle)
    assert torch.cuda.mem_get_info()[0] >= free0
    # the device still serves a normal handle
    h = capi.de_init(capi.make_config(16, 4, max_generations=3, target_error=0.0))
    try:
        assert capi.de_run(h)[0]["generations"] == 3
    finally:
        capi.de_destroy(h)


# ----------------------------------------------------------------------------- checkpoints
def test_checkpoint_of_another_problem_is_refused_before_any_copy(tmp_path):
    _need_gpu()
    d = 12
    o, M = problems.shift(d, seed=8), problems.rotation(d, seed=8)
    cfgs = [capi.make_config(64, d, objective=1, shift=o, rot=M, seed=5, run_id=r, max_generations=100,
                             target_error=0.0) for r in range(2)]
    h = capi.de_init_batch(cfgs)
    capi.de_step(h, 30)
    path = str(tmp_path / "ck.bin")
    capi.de_save(h, path)
    capi.de_destroy(h)
    changes = [dict(seed=6), dict(f=0.6), dict(cr=0.8), dict(shift=o + 1e-12), dict(rot=M[::-1].copy()),
               dict(objective=3), dict(lo=-99.0)]
    for ch in changes:
        # run 0 as saved, run 1 changed: the load must leave both runs as they were
        c1 = dict(np_=64, d=d, objective=1, shift=o, rot=M, seed=5, run_id=1, max_generations=100, target_error=0.0)
        c1.update(ch)
        h = capi.de_init_batch([cfgs[0], capi.make_config(**c1)])
        try:
            before = [capi.de_get_population(h, r) for r in range(2)]
            with pytest.raises(capi.DEError) as ei:
                capi.de_load(h, path)
            assert ei.value.status == capi.DE_ERR_STATE, ch
            after = [capi.de_get_population(h, r) for r in range(2)]
            for (xa, fa), (xb, fb) in zip(before, after):
                assert np.array_equal(xa, xb) and np.array_equal(fa, fb), ch
            assert capi.de_get_best(h, 0)["generations"] == 0
        finally:
            capi.de_destroy(h)
    # a new budget or target is not part of the problem: the checkpoint loads
    c0 = [capi.make_config(64, d, objective=1, shift=o, rot=M, seed=5, run_id=r, max_generations=500,
                           target_error=1e-3) for r in range(2)]
    h = capi.de_init_batch(c0)
    try:
        capi.de_load(h, path)
        assert capi.de_get_best(h, 1)["generations"] == 30
    finally:
        capi.de_destroy(h)
