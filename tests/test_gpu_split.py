"""GPU parity of the split-precision (BF16x3 / TF32x3 tcgen05) path against
the FP64 CPU oracle.

The trial construction is the FP64 one in every precision, so indices, masks
and trials must match the oracle bit for bit.  The split-precision fitness
must stay within the kernel's stated bound; every selection decision must
equal the oracle's outside the FP64 tolerance band, because comparisons the
split values cannot decide are redone in FP64.  Through the C ABI only.
"""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import capi, problems

pytestmark = pytest.mark.gpu

REL64 = 1e-12
# split-precision fitness tolerance relative to (|f| + S); S as defined by the
# oracle (term magnitudes plus first-order rounding of their inputs)
REL_SPLIT = {capi.DE_PREC_BF16X3: 1e-5, capi.DE_PREC_TF32X3: 1e-6}
PRECS = [capi.DE_PREC_BF16X3, capi.DE_PREC_TF32X3]


# the split-precision kernel paths: the persistent kernel as thread-block
# clusters (path 2) or with CTA-local products (path 4), and the three-kernel
# path (1); DE_GB300_PERSIST=0 disables both persistent forms,
# DE_GB300_PERSIST_MODE keeps one of them
PATH_ENV = {"cluster": ("1", "cluster"), "cta": ("1", "cta"), "three-kernel": ("0", "cta")}
PATH_NUM = {"cluster": 2, "cta": 4, "three-kernel": 1}


def _use_path(monkeypatch, name):
    persist, mode = PATH_ENV[name]
    monkeypatch.setenv("DE_GB300_PERSIST", persist)
    monkeypatch.setenv("DE_GB300_PERSIST_MODE", mode)


@pytest.fixture(params=["cluster", "cta", "three-kernel"])
def split_path(request, monkeypatch):
    """Run a test on every split-precision kernel path."""
    _use_path(monkeypatch, request.param)
    return request.param


def _check_path(h, split_path):
    """The handle runs the requested path where it applies (a persistent form
    falls back to the three-kernel path for shapes it does not cover)."""
    plan = capi.de_get_plan(h)
    assert plan["kernel_path"] in (1, PATH_NUM[split_path])
    return plan["kernel_path"] != 1


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("obj", [0, 1, 2, 3])
@pytest.mark.parametrize("d", [10, 100, 130, 300, 1000])
def test_split_eval_within_tolerance(prec, obj, d):
    torch = _need_gpu()
    if obj == 2 and d > 256:
        pytest.skip("split precision takes Rosenbrock up to d = 256")
    o = problems.shift(d, seed=2)
    M = problems.rotation(d, seed=2)
    X = problems.population(700, d, seed=3)
    X[:200] = o + np.random.default_rng(1).normal(size=(200, d)) * np.logspace(-5, 1, 200)[:, None]
    cfg = capi.make_config(64, d, objective=obj, shift=o, rot=M, precision=prec, max_generations=1)
    h = capi.de_init(cfg)
    try:
        xd = torch.from_numpy(X).cuda()
        fd = torch.zeros(len(X), dtype=torch.float64, device="cuda")
        capi.de_eval(h, 0, xd.data_ptr(), d, len(X), fd.data_ptr())
        torch.cuda.synchronize()
    finally:
        capi.de_destroy(h)
    f = fd.cpu().numpy()
    fo, sabs = oracle.evaluate(obj, X, o, M)
    err = np.abs(f - fo) / (np.abs(fo) + sabs)
    assert err.max() <= REL_SPLIT[prec], err.max()


@pytest.mark.parametrize("band", [capi.DE_BAND_ALL, capi.DE_BAND_NEAR])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize(
    "np_,d,obj,F,CR",
    [(1024, 100, 1, 0.5, 0.9), (64, 10, 0, 0.5, 0.9), (300, 37, 2, 0.8, 0.3), (130, 64, 3, 0.5, 1.0),
     (4, 1, 1, 0.5, 0.9),
     (200, 128, 1, 0.5, 0.9),    # the largest D of the CTA-local kernel: K fills the A operand's columns
     (96, 120, 0, 0.5, 0.9),     # K of 128 (BF16x3) and 120 (TF32x3)
     (256, 1000, 1, 0.5, 0.9),   # the large-dimension workload's D: four N tiles, K staged in chunks
     (130, 300, 3, 0.5, 0.9)],   # two N tiles, the second ragged
)
def test_split_generation_matches_oracle(prec, np_, d, obj, F, CR, split_path, band):
    _need_gpu()
    o = problems.shift(d, seed=7)
    M = problems.rotation(d, seed=7)
    X = problems.population(np_, d, seed=7)
    fX, _ = oracle.evaluate(obj, X, o, M)
    cfg = capi.make_config(np_, d, f=F, cr=CR, objective=obj, shift=o, rot=M, seed=7, precision=prec,
                           max_generations=10**6, target_error=0.0, debug_capture=True, fp64_band=band)
    h = capi.de_init(cfg)
    try:
        _check_path(h, split_path)
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, 4)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        xn, fn = capi.de_get_population(h)
        best = capi.de_get_best(h)
    finally:
        capi.de_destroy(h)
    r = oracle.step(X, fX, F, CR, -100, 100, obj, o, M, seed=7, generation=5)
    assert np.array_equal(g["idx"], r["idx"])
    assert np.array_equal(g["jrand"], r["jrand"])
    assert np.array_equal(g["mask"], r["mask"])
    assert np.array_equal(g["trial"], r["trial"])
    fp64 = g["fp64_checked"].astype(bool)
    scale = np.abs(r["f_trial"]) + r["sabs_trial"]
    tol = np.where(fp64, REL64, REL_SPLIT[prec]) * scale
    assert np.all(np.abs(g["f_trial"] - r["f_trial"]) <= tol)
    # with every undecidable comparison in FP64, decisions differ from the
    # oracle's only inside the FP64 band; with the near-optimum policy, also
    # inside the split-precision band of the trial (targets here are FP64)
    rel = REL64 if band == capi.DE_BAND_ALL else REL_SPLIT[prec]
    inband = np.abs(r["f_trial"] - fX) <= rel * scale
    assert np.array_equal(g["accept"][~inband], r["accept"][~inband])
    acc = g["accept"].astype(bool)
    assert np.array_equal(xn[acc], r["trial"][acc])
    assert np.array_equal(xn[~acc], X[~acc])
    # the best record is an FP64 value of the best individual
    b = best["best_index"]
    fo_b, sb = oracle.evaluate(obj, xn[b:b + 1], o, M)
    assert abs(best["best_f"] - fo_b[0]) <= REL64 * (abs(fo_b[0]) + sb[0])
    assert abs(best["best_f"] - r["f_next"].min()) <= REL64 * (abs(fo_b[0]) + sb[0])


@pytest.mark.parametrize("prec", PRECS)
def test_split_run_follows_the_fp64_trajectory(prec, split_path):
    """With the FP64 band deciding every comparison the split values cannot,
    the split-precision run of the small sphere workload takes the same
    decisions as the FP64 oracle: same population, same stop generation."""
    _need_gpu()
    d = 10
    o = problems.shift(d, seed=1)
    Xo, fo, go, evo, _ = oracle.run(64, d, 0.5, 0.9, -100, 100, 0, o, None, seed=1, max_generations=1000,
                                    target_error=1e-8)
    h = capi.de_init(capi.make_config(64, d, objective=0, shift=o, seed=1, precision=prec, max_generations=1000,
                                      target_error=1e-8, fp64_band=capi.DE_BAND_ALL))
    try:
        _check_path(h, split_path)
        res = capi.de_run(h)[0]
        x, f = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    assert res["generations"] == go and res["evals"] == evo
    assert np.array_equal(x, Xo)
    assert res["best_f"] < 1e-8


def test_persistent_path_is_used_for_the_rotated_rastrigin_workload(monkeypatch):
    """NP=1024, D=100 in split precision runs on a persistent kernel: the
    autotuner's choice of form, or the form DE_GB300_PERSIST_MODE keeps."""
    _need_gpu()
    d = 100
    o, M = problems.shift(d, seed=1), problems.rotation(d, seed=1)
    for mode, want in ((None, (2, 4)), ("cluster", (2,)), ("cta", (4,))):
        if mode is None:
            monkeypatch.delenv("DE_GB300_PERSIST_MODE", raising=False)
        else:
            monkeypatch.setenv("DE_GB300_PERSIST_MODE", mode)
        for prec in PRECS:
            h = capi.de_init(capi.make_config(1024, d, objective=1, shift=o, rot=M, precision=prec,
                                              max_generations=10))
            try:
                plan = capi.de_get_plan(h)
            finally:
                capi.de_destroy(h)
            assert plan["kernel_path"] in want, (mode, plan)
            assert plan["cluster_size"] == (8 if plan["kernel_path"] == 2 else 0), plan


@pytest.mark.parametrize("prec", PRECS)
def test_split_paths_agree_over_many_generations(prec, monkeypatch):
    """Both split kernel paths take the FP64 oracle's decisions, so their
    populations after 200 generations of the rotated Rastrigin workload at
    NP=300, D=30 are identical."""
    _need_gpu()
    d = 30
    o, M = problems.shift(d, seed=4), problems.rotation(d, seed=4)
    pops = []
    for name in ("cluster", "cta", "three-kernel"):
        _use_path(monkeypatch, name)
        h = capi.de_init(capi.make_config(300, d, objective=1, shift=o, rot=M, seed=3, precision=prec,
                                          max_generations=200, target_error=0.0, fp64_band=capi.DE_BAND_ALL))
        try:
            assert capi.de_get_plan(h)["kernel_path"] == PATH_NUM[name]
            capi.de_run(h)
            pops.append(capi.de_get_population(h))
        finally:
            capi.de_destroy(h)
    assert np.array_equal(pops[0][0], pops[1][0]) and np.array_equal(pops[0][0], pops[2][0])


def test_persistent_rows_per_cluster_do_not_change_results(monkeypatch):
    """The persistent kernel's rows per cluster (tuned at de_init) only change
    the tiling (NP = 120: 1 to 15 clusters): after 150 generations every
    tiling gives the same populations, fitness, counters and best records.
    With every undecidable comparison redone in FP64 the populations also
    equal the three-kernel path's; fitness kept from split-precision
    decisions agrees within the split tolerance (the two paths sum a row's
    FP32 terms in different orders)."""
    _need_gpu()
    d = 40
    o, M = problems.shift(d, seed=6), problems.rotation(d, seed=6)

    def run(persist, rows):
        monkeypatch.setenv("DE_GB300_PERSIST", "1" if persist else "0")
        monkeypatch.setenv("DE_GB300_PERSIST_MODE", "cluster")
        monkeypatch.setenv("DE_GB300_PERSIST_ROWS", rows)
        h = capi.de_init(capi.make_config(120, d, objective=3, shift=o, rot=M, seed=5, precision=capi.DE_PREC_BF16X3,
                                          max_generations=150, target_error=0.0, fp64_band=capi.DE_BAND_ALL))
        try:
            assert capi.de_get_plan(h)["kernel_path"] == (2 if persist else 1)
            capi.de_run(h)
            x, f = capi.de_get_population(h)
            return x, f, capi.de_get_best(h), capi.de_get_stats(h)
        finally:
            capi.de_destroy(h)

    ref = run(False, "128")
    tiled = [run(True, rows) for rows in ("8", "40", "88", "128")]
    keys = ("generations", "evals", "best_index", "stop_reason")
    for x, f, b, st in tiled:
        assert np.array_equal(x, tiled[0][0]) and np.array_equal(f, tiled[0][1])
        assert np.array_equal(b["best_x"], tiled[0][2]["best_x"]) and b["best_f"] == tiled[0][2]["best_f"]
        assert st == tiled[0][3]
        assert np.array_equal(x, ref[0])
        assert np.allclose(f, ref[1], rtol=1e-5, atol=0)
        for key in keys:
            assert b[key] == tiled[0][2][key] == ref[2][key], key
        assert st["trials"] == ref[3]["trials"] == 120 * 150  # trials evaluated since de_init


def test_cta_local_rows_per_cta_do_not_change_results(monkeypatch):
    """The CTA-local persistent kernel's targets per CTA only change the
    tiling (NP = 120: 8 to 120 CTAs): after 150 generations every tiling
    gives the same populations, fitness, counters and best records.  The
    populations also equal the cluster kernel's: both take every undecidable
    comparison in FP64.  Fitness kept from split-precision decisions agrees
    within the split tolerance (the two kernels group the tensor-core
    products of a coordinate differently)."""
    _need_gpu()
    d = 40
    o, M = problems.shift(d, seed=6), problems.rotation(d, seed=6)

    def run(mode, rows):
        monkeypatch.setenv("DE_GB300_PERSIST", "1")
        monkeypatch.setenv("DE_GB300_PERSIST_MODE", mode)
        monkeypatch.setenv("DE_GB300_PERSIST_ROWS" if mode == "cluster" else "DE_GB300_PERSIST_CTA_ROWS", rows)
        h = capi.de_init(capi.make_config(120, d, objective=3, shift=o, rot=M, seed=5, precision=capi.DE_PREC_BF16X3,
                                          max_generations=150, target_error=0.0, fp64_band=capi.DE_BAND_ALL))
        try:
            assert capi.de_get_plan(h)["kernel_path"] == PATH_NUM[mode]
            capi.de_run(h)
            x, f = capi.de_get_population(h)
            return x, f, capi.de_get_best(h), capi.de_get_stats(h)
        finally:
            capi.de_destroy(h)

    ref = run("cluster", "40")
    tiled = [run("cta", rows) for rows in ("1", "5", "8", "16")]
    for x, f, b, st in tiled:
        assert np.array_equal(x, tiled[0][0]) and np.array_equal(f, tiled[0][1])
        assert np.array_equal(b["best_x"], tiled[0][2]["best_x"]) and b["best_f"] == tiled[0][2]["best_f"]
        assert st == tiled[0][3]
        assert np.array_equal(x, ref[0])
        assert np.allclose(f, ref[1], rtol=1e-5, atol=0)
        for key in ("generations", "evals", "best_index", "stop_reason"):
            assert b[key] == ref[2][key], key
        assert st["trials"] == ref[3]["trials"] == 120 * 150


@pytest.mark.parametrize("prec", PRECS)
def test_near_policy_reaches_the_target_and_reports_fp64_best(prec):
    """With the default near-optimum policy the small sphere run still meets
    the 1e-8 target, and the reported best is the FP64 fitness of the best
    individual."""
    _need_gpu()
    d = 10
    o = problems.shift(d, seed=1)
    h = capi.de_init(capi.make_config(64, d, objective=0, shift=o, seed=1, precision=prec, max_generations=1000,
                                      target_error=1e-8))
    try:
        res = capi.de_run(h)[0]
        b = capi.de_get_best(h)
    finally:
        capi.de_destroy(h)
    assert res["stop_reason"] == capi.DE_STOP_TARGET and res["best_f"] < 1e-8
    fo, _ = oracle.evaluate(0, b["best_x"][None, :], o, None)
    assert abs(b["best_f"] - fo[0]) <= 1e-12 * max(abs(fo[0]), 1e-300) + 1e-30


@pytest.mark.parametrize("prec", PRECS)
def test_split_batch_of_mixed_widths_equals_single_runs(prec, monkeypatch):
    """A batch mixing runs of one and of several N tiles (D = 300 and D = 40)
    gives each run the population its own handle gives it (single runs on the
    same three-kernel path)."""
    _need_gpu()
    monkeypatch.setenv("DE_GB300_PERSIST", "0")
    shapes = [(150, 300, 1), (70, 40, 3), (200, 300, 0), (33, 40, 1)]
    cfgs = []
    for r, (n, d, obj) in enumerate(shapes):
        cfgs.append(capi.make_config(n, d, objective=obj, shift=problems.shift(d, seed=9, run_id=r),
                                     rot=problems.rotation(d, seed=9, run_id=r), seed=9, run_id=r, precision=prec,
                                     max_generations=12, target_error=0.0))
    h = capi.de_init_batch(cfgs)
    try:
        capi.de_step(h, 12)
        pops = [capi.de_get_population(h, r) for r in range(len(shapes))]
    finally:
        capi.de_destroy(h)
    for r, c in enumerate(cfgs):
        hs = capi.de_init(c)
        try:
            capi.de_step(hs, 12)
            xs, fs = capi.de_get_population(hs)
        finally:
            capi.de_destroy(hs)
        assert np.array_equal(pops[r][0], xs), r
        assert np.array_equal(pops[r][1], fs), r


def test_integer_fp32_rounding_equals_the_hardware_conversion():
    """The split operands are rounded to FP32 by integer operations; they must
    equal the GPU's round-to-nearest conversion bit for bit, ties included."""
    _need_gpu()
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2 ** 63, size=500_000, dtype=np.int64).astype(np.uint64)
    bits |= rng.integers(0, 2, size=bits.size).astype(np.uint64) << np.uint64(63)
    x = bits.view(np.float64)
    # values in the float range, exact halfway cases (both parities), the range edges
    f = rng.standard_normal(200_000).astype(np.float32) * np.float32(1e3)
    fb = f.view(np.uint32).astype(np.uint64)
    up = (fb + 1).astype(np.uint32).view(np.float32).astype(np.float64)
    ties = (f.astype(np.float64) + up) / 2
    edges = np.array([3.4028234663852886e38, 3.4028235677973366e38, 3.402823567797337e38, 1.1754943508222875e-38,
                      1.1754942106924411e-38, -1.1754943508222875e-38, 0.0, -0.0, np.inf, -np.inf, np.nan, 1e-320,
                      5e-324, 1e300, -1e300, 0.1, 1 / 3], dtype=np.float64)
    for arr in (x, ties, rng.uniform(-200, 200, 300_000), edges):
        assert capi.de_selftest_f32_rounding(arr) == 0


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("obj,d", [(1, 100), (3, 37)])
def test_split_generation_with_a_domain_scale_matches_oracle(prec, obj, d, split_path):
    """A domain scale other than 1 (y = (t - o) s, Sec. 7.3.1's folding of
    [-100, 100] onto the function's domain: 0.0512 for Rastrigin's +-5.12):
    the trial loops are compiled separately for a unit scale, so this case
    runs the other instance of each."""
    _need_gpu()
    np_, F, CR, s = 300, 0.5, 0.9, 0.0512
    o, M = problems.shift(d, seed=8), problems.rotation(d, seed=8)
    X = problems.population(np_, d, seed=8)
    fX, _ = oracle.evaluate(obj, X, o, M, scale=s)
    cfg = capi.make_config(np_, d, f=F, cr=CR, objective=obj, scale=s, shift=o, rot=M, seed=8, precision=prec,
                           max_generations=10**6, target_error=0.0, debug_capture=True, fp64_band=capi.DE_BAND_ALL)
    h = capi.de_init(cfg)
    try:
        _check_path(h, split_path)
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, 2)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        xn, _ = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    r = oracle.step(X, fX, F, CR, -100, 100, obj, o, M, seed=8, generation=3, scale=s)
    assert np.array_equal(g["trial"], r["trial"])
    fp64 = g["fp64_checked"].astype(bool)
    tol_scale = np.abs(r["f_trial"]) + r["sabs_trial"]
    assert np.all(np.abs(g["f_trial"] - r["f_trial"]) <= np.where(fp64, REL64, REL_SPLIT[prec]) * tol_scale)
    inband = np.abs(r["f_trial"] - fX) <= REL64 * tol_scale
    assert np.array_equal(g["accept"][~inband], r["accept"][~inband])
    acc = g["accept"].astype(bool)
    assert np.array_equal(xn[acc], r["trial"][acc]) and np.array_equal(xn[~acc], X[~acc])
