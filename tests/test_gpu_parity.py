"""GPU parity of the DE generation step against the FP64 CPU oracle.

Both sides get the same seeded inputs (population, shift, rotation, seed,
generation).  Indices, j_rand, crossover masks and trial vectors must match
bit for bit; fitness within tau = rel * (|f| + S_abs) with rel = 1e-12 (FP64),
S_abs the oracle's sum of term magnitudes; selection decisions must match
except where |f_trial - f_target| <= tau.  Everything goes through the C ABI.
"""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import capi, problems

pytestmark = pytest.mark.gpu

REL64 = 1e-12


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _bits(mask, d):
    return np.array([[(int(mask[i, j // 32]) >> (j % 32)) & 1 for j in range(d)] for i in range(mask.shape[0])],
                    dtype=bool)


def _problem(np_, d, obj, seed, rotate=True):
    o = problems.shift(d, seed=seed)
    M = problems.rotation(d, seed=seed) if rotate else None
    return o, M


@pytest.mark.parametrize("np_,d", [(64, 10), (5, 1), (33, 7), (1024, 100), (17, 130)])
def test_init_population_bit_exact(np_, d):
    _need_gpu()
    o, M = _problem(np_, d, 1, 3)
    cfg = capi.make_config(np_, d, objective=1, shift=o, rot=M, seed=123, run_id=2, max_generations=10)
    h = capi.de_init(cfg)
    try:
        x, f = capi.de_get_population(h)
        xo = oracle.init_population(np_, d, -100.0, 100.0, seed=123, run_id=2)
        assert np.array_equal(x, xo)
        fo, sabs = oracle.evaluate(1, xo, o, M)
        assert np.all(np.abs(f - fo) <= REL64 * (np.abs(fo) + sabs))
        b = capi.de_get_best(h)
        assert b["best_index"] == int(np.argmin(f))
        assert b["evals"] == np_ and b["generations"] == 0
        assert np.array_equal(b["best_x"], x[b["best_index"]])
    finally:
        capi.de_destroy(h)


@pytest.mark.parametrize("obj", [0, 1, 2, 3])
@pytest.mark.parametrize("d,rotate", [(1, False), (2, True), (10, True), (37, False), (100, True), (130, True)])
def test_eval_fp64_matches_oracle(obj, d, rotate):
    torch = _need_gpu()
    n = 300
    o, M = _problem(n, d, obj, 5 + d, rotate)
    X = problems.population(n, d, seed=9)
    # include the optimum and points near it
    X[0] = o
    X[1] = o + 1e-6
    cfg = capi.make_config(64, d, objective=obj, shift=o, rot=M, seed=1, max_generations=1)
    h = capi.de_init(cfg)
    try:
        xd = torch.from_numpy(X).cuda()
        fd = torch.zeros(n, dtype=torch.float64, device="cuda")
        capi.de_eval(h, 0, xd.data_ptr(), d, n, fd.data_ptr())
        torch.cuda.synchronize()
        f = fd.cpu().numpy()
        fo, sabs = oracle.evaluate(obj, X, o, M)
        err = np.abs(f - fo)
        tol = REL64 * (np.abs(fo) + sabs)
        assert np.all(err <= tol), (err / np.maximum(tol, 1e-300)).max()
    finally:
        capi.de_destroy(h)


def _step_compare(np_, d, obj, F, CR, seed, gen, rotate=True, lo=-100.0, hi=100.0, X=None):
    o, M = _problem(np_, d, obj, seed, rotate)
    if X is None:
        X = problems.population(np_, d, seed=seed, lo=lo, hi=hi)
    fX, _ = oracle.evaluate(obj, X, o, M)
    cfg = capi.make_config(np_, d, f=F, cr=CR, lo=lo, hi=hi, objective=obj, shift=o, rot=M, seed=seed,
                           max_generations=10**6, target_error=0.0, debug_capture=True)
    h = capi.de_init(cfg)
    try:
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, gen - 1)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        xn, fn = capi.de_get_population(h)
        best = capi.de_get_best(h)
    finally:
        capi.de_destroy(h)
    r = oracle.step(X, fX, F, CR, lo, hi, obj, o, M, seed=seed, generation=gen)
    assert np.array_equal(g["idx"], r["idx"])
    assert np.array_equal(g["jrand"], r["jrand"])
    assert np.array_equal(g["mask"], r["mask"])
    assert np.array_equal(g["trial"], r["trial"])
    tol = REL64 * (np.abs(r["f_trial"]) + r["sabs_trial"])
    assert np.all(np.abs(g["f_trial"] - r["f_trial"]) <= tol)
    band = np.abs(r["f_trial"] - fX) <= tol
    assert np.array_equal(g["accept"][~band], r["accept"][~band])
    acc = g["accept"].astype(bool)
    assert np.array_equal(xn[acc], r["trial"][acc])
    assert np.array_equal(xn[~acc], X[~acc])
    assert best["generations"] == gen
    assert best["best_index"] == int(np.argmin(fn))
    return g, r


@pytest.mark.parametrize(
    "np_,d,obj,F,CR,rotate",
    [
        (64, 10, 0, 0.5, 0.9, False),     # the small sphere workload
        (1024, 100, 1, 0.5, 0.9, True),   # the rotated Rastrigin workload
        (4, 1, 1, 0.5, 0.9, True),        # smallest population and dimension
        (37, 130, 2, 0.8, 0.3, True),     # ragged: two 128-coordinate chunks, odd tile
        (50, 33, 3, 0.5, 0.0, True),      # CR = 0: only j_rand crosses
        (50, 33, 1, 0.5, 1.0, False),     # CR = 1: every coordinate crosses
        (40, 16, 1, 1.9, 1.0, True),      # large F: bound repair on many coordinates
        (300, 50, 3, 0.0, 0.7, True),     # F = 0: mutant is x_r1
    ],
)
def test_one_generation_matches_oracle(np_, d, obj, F, CR, rotate):
    _need_gpu()
    g, r = _step_compare(np_, d, obj, F, CR, seed=7, gen=5, rotate=rotate)
    m = _bits(g["mask"], d)
    assert np.all(m.sum(axis=1) >= 1)


@pytest.mark.parametrize("lo,hi", [(-5.12, 5.12), (0.0, 1.0), (-100.0, 100.0)])
@pytest.mark.parametrize("F", [0.0, 0.5, 1.0])
def test_trials_on_and_next_to_the_bounds_match_oracle(lo, hi, F):
    """Mutants on a bound, one ulp either side of it, at signed zeros and
    subnormals: the kernels decide "inside" on the high 32 bits of the keys
    and only equal high words on all 64, so these are the cases where a
    wrong shortcut would show.  With F = 0 the mutant is x_r1 exactly."""
    _need_gpu()
    vals = [lo, hi, np.nextafter(lo, np.inf), np.nextafter(hi, -np.inf), np.nextafter(lo, -np.inf),
            np.nextafter(hi, np.inf), 0.0, -0.0, 5e-324, -5e-324, 1e-310, -1e-310, 0.5 * (lo + hi),
            hi + 2.0 ** -20 * abs(hi), lo - 2.0 ** -20 * max(abs(lo), 1.0), hi - 1e-12, lo + 1e-12]
    rng = np.random.default_rng(11)
    np_, d = 64, 24
    X = rng.choice(np.array(vals, dtype=np.float64), size=(np_, d))
    _step_compare(np_, d, 0, F, 1.0, seed=3, gen=2, rotate=True, lo=lo, hi=hi, X=X)


def test_trajectory_small_sphere_matches_oracle_run():
    """The FP64 sphere run (NP=64, D=10, F=0.5, CR=0.9, seed 1, up to 1000
    generations, stop at 1e-8): same stop generation, evaluations and best."""
    _need_gpu()
    d = 10
    o = problems.shift(d, seed=1)
    Xo, fo, go, evo, tro = oracle.run(64, d, 0.5, 0.9, -100, 100, 0, o, None, seed=1, max_generations=1000,
                                      target_error=1e-8, trace=True)
    cfg = capi.make_config(64, d, f=0.5, cr=0.9, objective=0, shift=o, seed=1, max_generations=1000,
                           target_error=1e-8)
    h = capi.de_init(cfg)
    try:
        res = capi.de_run(h)[0]
        x, f = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    assert res["generations"] == go
    assert res["evals"] == evo
    assert res["stop_reason"] == capi.DE_STOP_TARGET
    # sphere without rotation: the GPU sum order differs, so allow rounding
    assert np.array_equal(x, Xo)
    assert np.allclose(f, fo, rtol=1e-12, atol=0)


def test_batch_equals_single_runs_and_is_deterministic():
    _need_gpu()
    shapes = [(64, 10, 0), (100, 30, 1), (57, 50, 2), (200, 100, 3), (4, 3, 1)]
    cfgs = []
    for r, (np_, d, obj) in enumerate(shapes):
        o, M = _problem(np_, d, obj, 40 + r)
        cfgs.append(capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=1, run_id=r, max_generations=25,
                                     target_error=0.0))
    hb = capi.de_init_batch(cfgs)
    try:
        capi.de_run(hb, len(cfgs))
        batch = [capi.de_get_population(hb, r) for r in range(len(cfgs))]
    finally:
        capi.de_destroy(hb)
    for r, c in enumerate(cfgs):
        h = capi.de_init(c)
        try:
            capi.de_run(h)
            x, f = capi.de_get_population(h)
        finally:
            capi.de_destroy(h)
        assert np.array_equal(x, batch[r][0])
        assert np.array_equal(f, batch[r][1])


def test_checkpoint_split_run_equals_straight_run(tmp_path):
    _need_gpu()
    d = 20
    o, M = _problem(128, d, 1, 77)
    cfg = capi.make_config(128, d, objective=1, shift=o, rot=M, seed=5, max_generations=200, target_error=0.0)
    h = capi.de_init(cfg)
    capi.de_step(h, 200)
    x_straight, f_straight = capi.de_get_population(h)
    capi.de_destroy(h)
    h = capi.de_init(cfg)
    capi.de_step(h, 90)
    path = str(tmp_path / "ck.bin")
    capi.de_save(h, path)
    capi.de_destroy(h)
    h = capi.de_init(cfg)
    capi.de_load(h, path)
    capi.de_step(h, 110)
    x, f = capi.de_get_population(h)
    b = capi.de_get_best(h)
    capi.de_destroy(h)
    assert np.array_equal(x, x_straight) and np.array_equal(f, f_straight)
    assert b["generations"] == 200
    # a corrupted file is refused
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    open(path, "wb").write(bytes(raw))
    h = capi.de_init(cfg)
    try:
        with pytest.raises(capi.DEError) as ei:
            capi.de_load(h, path)
        assert ei.value.status == capi.DE_ERR_IO
    finally:
        capi.de_destroy(h)


def test_stop_rules():
    _need_gpu()
    d = 5
    o = problems.shift(d, seed=2)
    # max_generations = 0: nothing runs
    h = capi.de_init(capi.make_config(16, d, shift=o, max_generations=0))
    r = capi.de_run(h)[0]
    capi.de_destroy(h)
    assert r["generations"] == 0 and r["stop_reason"] == capi.DE_STOP_GENERATIONS and r["evals"] == 16
    # evaluation budget: stops at the first generation with evals >= budget
    h = capi.de_init(capi.make_config(16, d, shift=o, max_evals=16 * 11 + 3, max_generations=10**6,
                                      target_error=0.0))
    r = capi.de_run(h)[0]
    capi.de_destroy(h)
    assert r["stop_reason"] == capi.DE_STOP_EVALS and r["generations"] == 11 and r["evals"] == 16 * 12
    # best never increases across generations
    h = capi.de_init(capi.make_config(32, d, objective=1, shift=o, max_generations=10**6, target_error=0.0))
    last = np.inf
    for _ in range(30):
        capi.de_step(h, 1)
        b = capi.de_get_best(h)["best_f"]
        assert b <= last
        last = b
    capi.de_destroy(h)
