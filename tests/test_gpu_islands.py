"""GPU parity of the island model (Sec. 3.2, Sec. 5.4) against the CPU
oracle, through the C ABI: island populations after ring migrations, jDE
parameters carried by migrants, and the model's common stop; the same for
asynchronous migration (migrants one interval late, through a mailbox)."""
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


# the FP64 forms an island model runs on: one kernel per generation with the
# migration kernels between generations (path 0), or the cooperative kernel
# migrating inside its generation loop (path 3)
FP64_FORMS = [("0", 0), ("1", 3)]


@pytest.fixture(params=FP64_FORMS, ids=["per_generation", "cooperative"])
def fp64_form(request, monkeypatch):
    env, path = request.param
    monkeypatch.setenv("DE_GB300_FP64_PERSIST", env)
    # the heuristic tile size (no timed choice from an earlier test's cache),
    # with which every tile of these shapes is resident at once
    monkeypatch.setenv("DE_GB300_AUTOTUNE", "0")
    return path


def _run(m, interval, nmig, np_, d, obj, G, target=0.0, rotate=True, seed=3, asynchronous=False, path=None, **kw):
    o = problems.shift(d, seed=seed)
    M = problems.rotation(d, seed=seed) if rotate else None
    cfg = capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=seed, run_id=5, max_generations=G,
                           target_error=target, **kw)
    h = capi.de_init_islands_ex(cfg, m, interval, nmig,
                                capi.DE_MIGRATE_ASYNC if asynchronous else capi.DE_MIGRATE_SYNC)
    try:
        if path is not None:
            assert capi.de_get_plan(h)["kernel_path"] == path
        res = capi.de_run(h, m)
        pops = [capi.de_get_population(h, k) for k in range(m)]
        ad = [capi.de_get_adaptive(h, k) for k in range(m)] if kw.get("jde") else None
    finally:
        capi.de_destroy(h)
    Xo, fo, go, evo, Fo, Co = oracle.run_islands(m, interval, nmig, np_, d, 0.5, 0.9, -100, 100, obj, o, M,
                                                 seed=seed, max_generations=G, target_error=target, run_id=5,
                                                 strategy=kw.get("strategy", 0), jde=kw.get("jde", False),
                                                 asynchronous=asynchronous)
    return res, pops, ad, (Xo, fo, go, evo, Fo, Co), (o, M)


@pytest.mark.parametrize("m,interval,nmig,np_,d,obj", [(4, 5, 2, 32, 10, 1), (3, 1, 1, 20, 7, 3), (8, 7, 3, 50, 30, 2)])
def test_island_populations_match_oracle(m, interval, nmig, np_, d, obj, fp64_form):
    _need_gpu()
    G = 40
    res, pops, _, (Xo, fo, go, evo, _, _), (o, M) = _run(m, interval, nmig, np_, d, obj, G, path=fp64_form)
    assert all(r["generations"] == G for r in res)
    for k in range(m):
        x, f = pops[k]
        assert np.array_equal(x, Xo[k])
        _, sabs = oracle.evaluate(obj, x, o, M)
        assert np.all(np.abs(f - fo[k]) <= 1e-12 * (np.abs(fo[k]) + sabs))


def test_jde_islands_carry_parameters_like_the_oracle(fp64_form):
    _need_gpu()
    m, G = 4, 30
    res, pops, ad, (Xo, fo, go, evo, Fo, Co), _ = _run(m, 3, 2, 24, 12, 1, G, jde=True, strategy=capi.DE_RAND1EXP,
                                                      path=fp64_form)
    for k in range(m):
        assert np.array_equal(pops[k][0], Xo[k])
        assert np.array_equal(ad[k][0], Fo[k]) and np.array_equal(ad[k][1], Co[k])


def test_the_model_stops_together_at_the_oracles_generation(fp64_form):
    _need_gpu()
    m = 4
    res, pops, _, (Xo, fo, go, evo, _, _), _ = _run(m, 10, 1, 32, 5, 0, 3000, target=1e-8, rotate=False,
                                                   path=fp64_form)
    assert all(r["generations"] == go for r in res)
    assert all(r["stop_reason"] == capi.DE_STOP_TARGET for r in res)
    assert min(r["best_f"] for r in res) < 1e-8
    for k in range(m):
        assert np.array_equal(pops[k][0], Xo[k])


def test_reset_replays_the_same_island_run():
    _need_gpu()
    o = problems.shift(10, seed=1)
    cfg = capi.make_config(24, 10, objective=1, shift=o, seed=2, max_generations=25, target_error=0.0)
    h = capi.de_init_islands(cfg, 3, 4, 2)
    try:
        capi.de_run(h, 3)
        a = [capi.de_get_population(h, k) for k in range(3)]
        capi.de_reset(h)
        capi.de_run(h, 3)
        b = [capi.de_get_population(h, k) for k in range(3)]
    finally:
        capi.de_destroy(h)
    for k in range(3):
        assert np.array_equal(a[k][0], b[k][0]) and np.array_equal(a[k][1], b[k][1])


# ----------------------------------------------------------------- asynchronous
@pytest.mark.parametrize("m,interval,nmig,np_,d,obj", [(4, 5, 2, 32, 10, 1), (3, 1, 1, 20, 7, 3), (8, 7, 3, 50, 30, 2),
                                                       (2, 3, 4, 16, 5, 0)])
def test_async_island_populations_match_oracle(m, interval, nmig, np_, d, obj, fp64_form):
    _need_gpu()
    G = 40
    res, pops, _, (Xo, fo, go, evo, _, _), (o, M) = _run(m, interval, nmig, np_, d, obj, G, asynchronous=True,
                                                         path=fp64_form)
    assert all(r["generations"] == G for r in res)
    for k in range(m):
        x, f = pops[k]
        assert np.array_equal(x, Xo[k])
        _, sabs = oracle.evaluate(obj, x, o, M)
        assert np.all(np.abs(f - fo[k]) <= 1e-12 * (np.abs(fo[k]) + sabs))


def test_async_differs_from_sync_on_the_gpu_as_in_the_oracle():
    _need_gpu()
    a = _run(4, 4, 2, 24, 8, 1, 20, asynchronous=True)
    b = _run(4, 4, 2, 24, 8, 1, 20)
    assert any(not np.array_equal(a[1][k][0], b[1][k][0]) for k in range(4))
    for k in range(4):
        assert np.array_equal(a[1][k][0], a[3][0][k]) and np.array_equal(b[1][k][0], b[3][0][k])


def test_async_jde_islands_carry_parameters_like_the_oracle(fp64_form):
    _need_gpu()
    m, G = 4, 30
    res, pops, ad, (Xo, fo, go, evo, Fo, Co), _ = _run(m, 3, 2, 24, 12, 1, G, jde=True, strategy=capi.DE_RAND1EXP,
                                                      asynchronous=True, path=fp64_form)
    for k in range(m):
        assert np.array_equal(pops[k][0], Xo[k])
        assert np.array_equal(ad[k][0], Fo[k]) and np.array_equal(ad[k][1], Co[k])


def test_async_model_stops_together_at_the_oracles_generation(fp64_form):
    _need_gpu()
    m = 4
    res, pops, _, (Xo, fo, go, evo, _, _), _ = _run(m, 10, 1, 32, 5, 0, 3000, target=1e-8, rotate=False,
                                                   asynchronous=True, path=fp64_form)
    assert all(r["generations"] == go for r in res)
    assert all(r["stop_reason"] == capi.DE_STOP_TARGET for r in res)
    for k in range(m):
        assert np.array_equal(pops[k][0], Xo[k])


def test_async_reset_empties_the_mailbox_and_replays_the_run():
    """de_reset forgets the posts: the replay takes no migrants at the first
    migration point after it, exactly as the first run did."""
    _need_gpu()
    o = problems.shift(10, seed=1)
    cfg = capi.make_config(24, 10, objective=1, shift=o, seed=2, max_generations=25, target_error=0.0)
    h = capi.de_init_islands_ex(cfg, 3, 4, 2, capi.DE_MIGRATE_ASYNC)
    try:
        capi.de_run(h, 3)
        a = [capi.de_get_population(h, k) for k in range(3)]
        capi.de_reset(h)
        capi.de_run(h, 3)
        b = [capi.de_get_population(h, k) for k in range(3)]
    finally:
        capi.de_destroy(h)
    Xo = oracle.run_islands(3, 4, 2, 24, 10, 0.5, 0.9, -100, 100, 1, o, None, seed=2, max_generations=25,
                            target_error=0.0, asynchronous=True)[0]
    for k in range(3):
        assert np.array_equal(a[k][0], b[k][0]) and np.array_equal(a[k][1], b[k][1])
        assert np.array_equal(a[k][0], Xo[k])


def test_async_islands_stepped_across_launches_match_oracle(fp64_form):
    """Generations in steps of 7 with migrations every 5: the mailbox's posts
    and the point of the last post carry over from one launch to the next."""
    _need_gpu()
    m, interval, nmig, np_, d, obj, G = 4, 5, 2, 24, 8, 1, 42
    o, M = problems.shift(d, seed=7), problems.rotation(d, seed=7)
    cfg = capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=7, run_id=2, max_generations=10**6,
                           target_error=0.0)
    h = capi.de_init_islands_ex(cfg, m, interval, nmig, capi.DE_MIGRATE_ASYNC)
    try:
        assert capi.de_get_plan(h)["kernel_path"] == fp64_form
        for _ in range(G // 7):
            capi.de_step(h, 7)
        pops = [capi.de_get_population(h, k)[0] for k in range(m)]
    finally:
        capi.de_destroy(h)
    Xo = oracle.run_islands(m, interval, nmig, np_, d, 0.5, 0.9, -100, 100, obj, o, M, seed=7, max_generations=G,
                            target_error=0.0, run_id=2, asynchronous=True)[0]
    for k in range(m):
        assert np.array_equal(pops[k], Xo[k])
