"""GPU parity of the DE strategy variants (DE/best/1/bin, DE/rand/1/exp) and
jDE's self-adaptive F and CR (Sec. 2) against the FP64 CPU oracle, through
the C ABI.  Indices, j_rand, masks, trials and the jDE parameters of the next
generation are compared bit for bit; fitness within 1e-12 of the term
magnitudes; selection outside that band."""
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


def _step(np_, d, obj, F, CR, strategy, jde, seed=7, gen=5, rotate=True, jF=None, jCR=None, X=None, fX=None):
    o = problems.shift(d, seed=seed)
    M = problems.rotation(d, seed=seed) if rotate else None
    if X is None:
        X = problems.population(np_, d, seed=seed)
    if fX is None:
        fX, _ = oracle.evaluate(obj, X, o, M)
    cfg = capi.make_config(np_, d, f=F, cr=CR, objective=obj, shift=o, rot=M, seed=seed, max_generations=10**6,
                           target_error=0.0, debug_capture=True, strategy=strategy, jde=jde)
    h = capi.de_init(cfg)
    try:
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, gen - 1)
        if jde and (jF is not None or jCR is not None):
            capi.de_set_adaptive(h, 0, jF, jCR)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        xn, fn = capi.de_get_population(h)
        ad = capi.de_get_adaptive(h) if jde else None
    finally:
        capi.de_destroy(h)
    r = oracle.step(X, fX, F, CR, -100, 100, obj, o, M, seed=seed, generation=gen, strategy=strategy, jde=jde,
                    jF=jF, jCR=jCR)
    assert np.array_equal(g["idx"], r["idx"])
    assert np.array_equal(g["jrand"], r["jrand"])
    assert np.array_equal(g["mask"], r["mask"])
    assert np.array_equal(g["trial"], r["trial"])
    tol = REL64 * (np.abs(r["f_trial"]) + r["sabs_trial"])
    assert np.all(np.abs(g["f_trial"] - r["f_trial"]) <= tol)
    band = np.abs(r["f_trial"] - fX) <= tol
    assert np.array_equal(g["accept"][~band], r["accept"][~band])
    acc = g["accept"].astype(bool)
    assert np.array_equal(xn[acc], r["trial"][acc]) and np.array_equal(xn[~acc], X[~acc])
    if jde:
        same = g["accept"] == r["accept"]
        assert np.array_equal(ad[0][same], r["F_next"][same])
        assert np.array_equal(ad[1][same], r["CR_next"][same])
    return g, r, ad


@pytest.mark.parametrize("strategy", [capi.DE_BEST1BIN, capi.DE_RAND1EXP])
@pytest.mark.parametrize(
    "np_,d,obj,F,CR,rotate",
    [
        (64, 10, 0, 0.5, 0.9, False),
        (256, 100, 1, 0.5, 0.9, True),
        (37, 130, 2, 0.8, 0.3, True),    # two 128-coordinate chunks, ragged tail
        (50, 33, 3, 0.5, 0.0, True),     # CR = 0: exp block of length 1
        (50, 300, 1, 0.5, 1.0, False),   # CR = 1: exp length d, scan over three chunks
        (40, 16, 1, 1.9, 0.95, True),    # bound repair on many coordinates
        (4, 1, 1, 0.5, 0.9, True),       # smallest population and dimension
    ],
)
def test_strategy_one_generation_matches_oracle(strategy, np_, d, obj, F, CR, rotate):
    _need_gpu()
    g, r, _ = _step(np_, d, obj, F, CR, strategy, False, rotate=rotate)
    m = _bits(g["mask"], d)
    assert np.all(m.sum(axis=1) >= 1)
    if strategy == capi.DE_RAND1EXP and CR == 1.0:
        assert m.all()


def test_exp_block_lengths_span_chunk_boundaries():
    """CR close to 1 at d = 400: block lengths reach past 128 and 256."""
    _need_gpu()
    g, r, _ = _step(300, 400, 0, 0.5, 0.995, capi.DE_RAND1EXP, False, rotate=False)
    L = _bits(g["mask"], 400).sum(axis=1)
    assert L.max() > 128 and L.min() >= 1


def test_best1bin_base_follows_ties_and_lowest_index():
    _need_gpu()
    np_, d = 40, 7
    X = problems.population(np_, d, seed=1)
    fX, _ = oracle.evaluate(0, X)
    fX[5] = fX[9] = fX.min() - 1.0
    g, r, _ = _step(np_, d, 0, 0.0, 1.0, capi.DE_BEST1BIN, False, rotate=False, X=X, fX=fX)
    assert np.all(g["trial"] == X[5])


@pytest.mark.parametrize("strategy", [capi.DE_RAND1BIN, capi.DE_BEST1BIN, capi.DE_RAND1EXP])
@pytest.mark.parametrize("np_,d,obj,rotate", [(64, 10, 0, False), (1024, 100, 1, True), (77, 129, 3, True)])
def test_jde_one_generation_matches_oracle(strategy, np_, d, obj, rotate):
    _need_gpu()
    rng = np.random.default_rng(11)
    jF = 0.1 + 0.9 * rng.random(np_)
    jCR = rng.random(np_)
    g, r, ad = _step(np_, d, obj, 0.5, 0.9, strategy, True, rotate=rotate, jF=jF, jCR=jCR)
    acc = g["accept"].astype(bool)
    assert np.array_equal(ad[0][~acc], jF[~acc]) and np.array_equal(ad[1][~acc], jCR[~acc])


@pytest.mark.parametrize("strategy,jde", [(capi.DE_BEST1BIN, False), (capi.DE_RAND1EXP, False),
                                          (capi.DE_RAND1BIN, True), (capi.DE_RAND1EXP, True)])
def test_variant_trajectory_small_sphere_matches_oracle_run(strategy, jde):
    """200 generations of the small sphere (NP = 64, D = 10): the same
    populations, fitness (the sphere without rotation sums in another order:
    rounding only) and jDE parameters."""
    _need_gpu()
    d, G = 10, 200
    o = problems.shift(d, seed=1)
    res = oracle.run(64, d, 0.5, 0.9, -100, 100, 0, o, None, seed=1, max_generations=G, target_error=0.0,
                     strategy=strategy, jde=jde, return_adaptive=True)
    Xo, fo, go = res[0], res[1], res[2]
    cfg = capi.make_config(64, d, objective=0, shift=o, seed=1, max_generations=G, target_error=0.0,
                           strategy=strategy, jde=jde)
    h = capi.de_init(cfg)
    try:
        out = capi.de_run(h)[0]
        x, f = capi.de_get_population(h)
        ad = capi.de_get_adaptive(h) if jde else None
    finally:
        capi.de_destroy(h)
    assert out["generations"] == go == G
    assert np.array_equal(x, Xo)
    assert np.allclose(f, fo, rtol=1e-12, atol=0)
    if jde:
        assert np.array_equal(ad[0], res[5]) and np.array_equal(ad[1], res[6])


def test_batch_of_mixed_strategies_equals_single_runs():
    _need_gpu()
    specs = [(64, 10, 0, 0, False), (100, 30, 1, 1, False), (57, 50, 2, 2, True), (200, 100, 3, 0, True),
             (48, 20, 1, 0, False)]
    cfgs = []
    for r, (np_, d, obj, st, jde) in enumerate(specs):
        o, M = problems.shift(d, seed=40 + r), problems.rotation(d, seed=40 + r)
        cfgs.append(capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=1, run_id=r, max_generations=25,
                                     target_error=0.0, strategy=st, jde=jde))
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
        assert np.array_equal(x, batch[r][0]) and np.array_equal(f, batch[r][1])


def test_jde_checkpoint_and_generation_parity(tmp_path):
    """A jDE run saved after 40 generations and resumed equals the straight
    run, F_i and CR_i included; moving the generation counter to the other
    buffer parity keeps them."""
    _need_gpu()
    d = 20
    o, M = problems.shift(d, seed=9), problems.rotation(d, seed=9)
    cfg = capi.make_config(96, d, objective=1, shift=o, rot=M, seed=3, max_generations=100, target_error=0.0,
                           strategy=capi.DE_RAND1EXP, jde=True)
    h = capi.de_init(cfg)
    capi.de_step(h, 100)
    xs, fs = capi.de_get_population(h)
    ads = capi.de_get_adaptive(h)
    capi.de_destroy(h)
    h = capi.de_init(cfg)
    capi.de_step(h, 40)
    path = str(tmp_path / "jde.bin")
    capi.de_save(h, path)
    capi.de_destroy(h)
    h = capi.de_init(cfg)
    try:
        capi.de_load(h, path)
        capi.de_step(h, 60)
        x, f = capi.de_get_population(h)
        ad = capi.de_get_adaptive(h)
        a0 = capi.de_get_adaptive(h)
        capi.de_set_generation(h, 0, 101)
        a1 = capi.de_get_adaptive(h)
    finally:
        capi.de_destroy(h)
    assert np.array_equal(x, xs) and np.array_equal(f, fs)
    assert np.array_equal(ad[0], ads[0]) and np.array_equal(ad[1], ads[1])
    assert np.array_equal(a0[0], a1[0]) and np.array_equal(a0[1], a1[1])


def test_adaptive_getters_reject_plain_runs_and_bad_values():
    _need_gpu()
    h = capi.de_init(capi.make_config(16, 5, max_generations=10))
    try:
        with pytest.raises(capi.DEError) as ei:
            capi.de_get_adaptive(h)
        assert ei.value.status == capi.DE_ERR_STATE
    finally:
        capi.de_destroy(h)
    h = capi.de_init(capi.make_config(16, 5, max_generations=10, jde=True, f=0.7, cr=0.2))
    try:
        F, CR = capi.de_get_adaptive(h)
        assert np.all(F == 0.7) and np.all(CR == 0.2)
        with pytest.raises(capi.DEError) as ei:
            capi.de_set_adaptive(h, 0, np.full(16, 2.5), None)
        assert ei.value.status == capi.DE_ERR_INVALID_ARG
        with pytest.raises(capi.DEError) as ei:
            capi.de_set_adaptive(h, 0, None, np.full(16, -0.1))
        assert ei.value.status == capi.DE_ERR_INVALID_ARG
    finally:
        capi.de_destroy(h)


# ------------------------------------------------------------------ split precisions
REL_SPLIT = {capi.DE_PREC_BF16X3: 1e-5, capi.DE_PREC_TF32X3: 1e-6}


# split-precision kernel paths: persistent clusters (2), persistent with
# CTA-local products (4), three kernels (1)
PATH_ENV = {"cluster": ("1", "cluster"), "cta": ("1", "cta"), "three-kernel": ("0", "cta")}


def _use_path(monkeypatch, name):
    monkeypatch.setenv("DE_GB300_PERSIST", PATH_ENV[name][0])
    monkeypatch.setenv("DE_GB300_PERSIST_MODE", PATH_ENV[name][1])


@pytest.fixture(params=["cluster", "cta", "three-kernel"])
def split_path(request, monkeypatch):
    _use_path(monkeypatch, request.param)
    return request.param


@pytest.mark.parametrize("prec", [capi.DE_PREC_BF16X3, capi.DE_PREC_TF32X3])
@pytest.mark.parametrize("strategy,jde", [(capi.DE_BEST1BIN, False), (capi.DE_RAND1EXP, False),
                                          (capi.DE_RAND1BIN, True), (capi.DE_RAND1EXP, True),
                                          (capi.DE_BEST1BIN, True)])
@pytest.mark.parametrize("np_,d,obj", [(256, 100, 1), (70, 37, 3), (1024, 100, 1)])
def test_split_variants_one_generation_match_oracle(prec, strategy, jde, np_, d, obj, split_path):
    _need_gpu()
    o, M = problems.shift(d, seed=21), problems.rotation(d, seed=21)
    X = problems.population(np_, d, seed=21)
    fX, _ = oracle.evaluate(obj, X, o, M)
    rng = np.random.default_rng(21)
    jF = 0.1 + 0.9 * rng.random(np_) if jde else None
    jCR = rng.random(np_) if jde else None
    cfg = capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=21, precision=prec, max_generations=10**6,
                           target_error=0.0, debug_capture=True, fp64_band=capi.DE_BAND_ALL, strategy=strategy,
                           jde=jde)
    h = capi.de_init(cfg)
    try:
        plan = capi.de_get_plan(h)["kernel_path"]
        assert plan in {"cluster": (1, 2), "cta": (1, 4), "three-kernel": (1,)}[split_path]
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, 8)
        if jde:
            capi.de_set_adaptive(h, 0, jF, jCR)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        xn, fn = capi.de_get_population(h)
        ad = capi.de_get_adaptive(h) if jde else None
    finally:
        capi.de_destroy(h)
    r = oracle.step(X, fX, 0.5, 0.9, -100, 100, obj, o, M, seed=21, generation=9, strategy=strategy, jde=jde,
                    jF=jF, jCR=jCR)
    assert np.array_equal(g["idx"], r["idx"]) and np.array_equal(g["jrand"], r["jrand"])
    assert np.array_equal(g["mask"], r["mask"]) and np.array_equal(g["trial"], r["trial"])
    fp64 = g["fp64_checked"].astype(bool)
    scale = np.abs(r["f_trial"]) + r["sabs_trial"]
    assert np.all(np.abs(g["f_trial"] - r["f_trial"]) <= np.where(fp64, REL64, REL_SPLIT[prec]) * scale)
    inband = np.abs(r["f_trial"] - fX) <= REL64 * scale
    assert np.array_equal(g["accept"][~inband], r["accept"][~inband])
    acc = g["accept"].astype(bool)
    assert np.array_equal(xn[acc], r["trial"][acc]) and np.array_equal(xn[~acc], X[~acc])
    if jde:
        same = g["accept"] == r["accept"]
        assert np.array_equal(ad[0][same], r["F_next"][same]) and np.array_equal(ad[1][same], r["CR_next"][same])


@pytest.mark.parametrize("strategy,jde", [(capi.DE_BEST1BIN, False), (capi.DE_RAND1EXP, True)])
def test_split_variant_paths_agree_over_many_generations(strategy, jde, monkeypatch):
    """With every undecidable comparison in FP64 both split kernel paths take
    the same decisions: identical populations and jDE parameters after 150
    generations."""
    _need_gpu()
    d = 30
    o, M = problems.shift(d, seed=4), problems.rotation(d, seed=4)
    out = []
    for name in ("cluster", "cta", "three-kernel"):
        _use_path(monkeypatch, name)
        h = capi.de_init(capi.make_config(300, d, objective=1, shift=o, rot=M, seed=3, precision=capi.DE_PREC_BF16X3,
                                          max_generations=150, target_error=0.0, fp64_band=capi.DE_BAND_ALL,
                                          strategy=strategy, jde=jde))
        try:
            capi.de_run(h)
            out.append((capi.de_get_population(h), capi.de_get_adaptive(h) if jde else None))
        finally:
            capi.de_destroy(h)
    for k in (1, 2):
        assert np.array_equal(out[0][0][0], out[k][0][0])
        if jde:
            assert np.array_equal(out[0][1][0], out[k][1][0]) and np.array_equal(out[0][1][1], out[k][1][1])


def test_split_batch_with_variants_equals_single_runs(monkeypatch):
    _need_gpu()
    monkeypatch.setenv("DE_GB300_PERSIST", "0")
    specs = [(64, 10, 0, 1, False), (100, 30, 1, 2, True), (57, 50, 3, 0, True)]
    cfgs = []
    for r, (np_, d, obj, st, jde) in enumerate(specs):
        o, M = problems.shift(d, seed=60 + r), problems.rotation(d, seed=60 + r)
        cfgs.append(capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=1, run_id=r, max_generations=25,
                                     target_error=0.0, precision=capi.DE_PREC_BF16X3, fp64_band=capi.DE_BAND_ALL,
                                     strategy=st, jde=jde))
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
