"""GPU parity of the proposed benchmark's functions (Sec. 7.3, Table 2:
basic, hybrid and composition functions) on the FP64 path against the CPU
oracle, through the C ABI: evaluations within 1e-12 (|f| + S), and whole
generations with bit-exact trials and selections outside that band."""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import capi, problems

pytestmark = pytest.mark.gpu

REL64 = 1e-12
BASIC = list(range(5, 15))
HYBRID = [15, 16, 17]
COMPOSITION = [18, 19, 20]


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _data(obj, d, seed, rotate=True):
    s = problems.suite(obj, d, seed=seed)
    perm = s["perm"]
    scale = 1.0 if obj in HYBRID + COMPOSITION else 0.05
    return s["shift"], (s["rot"] if rotate else None), perm, scale


def _eval_compare(obj, d, rotate=True, n=200, seed=3):
    torch = _need_gpu()
    o, M, perm, scale = _data(obj, d, seed, rotate)
    X = problems.population(n, d, seed=seed + 1)
    # the optimum (and each component's optimum) and points near them
    if obj in COMPOSITION:
        for c in range(o.shape[0]):
            X[2 * c] = o[c]
            X[2 * c + 1] = o[c] + 1e-6
    else:
        X[0] = o
        X[1] = o + 1e-6
    cfg = capi.make_config(16, d, objective=obj, shift=o, rot=M, perm=perm, scale=scale, seed=1, max_generations=1)
    h = capi.de_init(cfg)
    try:
        xd = torch.from_numpy(X).cuda()
        fd = torch.zeros(n, dtype=torch.float64, device="cuda")
        capi.de_eval(h, 0, xd.data_ptr(), d, n, fd.data_ptr())
        torch.cuda.synchronize()
        f = fd.cpu().numpy()
    finally:
        capi.de_destroy(h)
    fo, sabs = oracle.evaluate(obj, X, o, M, scale=scale, perm=perm)
    err = np.abs(f - fo)
    tol = REL64 * (np.abs(fo) + sabs)
    assert np.all(err <= tol), (obj, d, (err / np.maximum(tol, 1e-300)).max())
    return f, fo, X, o


@pytest.mark.parametrize("obj", BASIC)
@pytest.mark.parametrize("d,rotate", [(1, False), (2, True), (10, True), (37, False), (100, True)])
def test_basic_functions_match_oracle(obj, d, rotate):
    _eval_compare(obj, d, rotate)


@pytest.mark.parametrize("obj", HYBRID)
@pytest.mark.parametrize("d,rotate", [(10, True), (30, True), (37, False), (50, True), (100, True)])
def test_hybrid_functions_match_oracle(obj, d, rotate):
    f, fo, X, o = _eval_compare(obj, d, rotate)
    assert abs(f[0]) <= 1e-9  # x = o


@pytest.mark.parametrize("obj", COMPOSITION)
@pytest.mark.parametrize("d,rotate", [(2, True), (10, True), (30, True), (37, False), (100, True)])
def test_composition_functions_match_oracle(obj, d, rotate):
    f, fo, X, o = _eval_compare(obj, d, rotate)
    # at x = o_c the composition takes bias_c (plus lambda_c g_c(0), zero up to rounding)
    bias = {18: [0, 100, 200], 19: [0, 100, 200, 300], 20: [0, 100, 200, 300, 400]}[obj]
    for c, b in enumerate(bias):
        assert abs(f[2 * c] - b) <= 1e-9


@pytest.mark.parametrize("obj", BASIC + HYBRID + COMPOSITION)
def test_suite_one_generation_matches_oracle(obj):
    _need_gpu()
    np_, d = 96, 30
    o, M, perm, scale = _data(obj, d, 11)
    X = problems.population(np_, d, seed=12)
    fX, _ = oracle.evaluate(obj, X, o, M, scale=scale, perm=perm)
    cfg = capi.make_config(np_, d, objective=obj, shift=o, rot=M, perm=perm, scale=scale, seed=13,
                           max_generations=100, target_error=0.0, debug_capture=True)
    h = capi.de_init(cfg)
    try:
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, 6)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        xn, fn = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    r = oracle.step(X, fX, 0.5, 0.9, -100, 100, obj, o, M, seed=13, generation=7, scale=scale, perm=perm)
    assert np.array_equal(g["trial"], r["trial"])
    tol = REL64 * (np.abs(r["f_trial"]) + r["sabs_trial"])
    assert np.all(np.abs(g["f_trial"] - r["f_trial"]) <= tol)
    band = np.abs(r["f_trial"] - fX) <= tol
    assert np.array_equal(g["accept"][~band], r["accept"][~band])
    acc = g["accept"].astype(bool)
    assert np.array_equal(xn[acc], r["trial"][acc]) and np.array_equal(xn[~acc], X[~acc])


@pytest.mark.parametrize("obj", [15, 18, 20])
def test_suite_trajectory_matches_oracle_run(obj):
    """60 generations of a D = 10 run from the library's own initial
    population: the same populations as the oracle's run."""
    _need_gpu()
    d, G = 10, 60
    o, M, perm, scale = _data(obj, d, 21)
    Xo, fo, go, _, _ = oracle.run(48, d, 0.5, 0.9, -100, 100, obj, o, M, seed=22, max_generations=G,
                                  target_error=0.0, scale=scale, perm=perm)
    cfg = capi.make_config(48, d, objective=obj, shift=o, rot=M, perm=perm, scale=scale, seed=22, max_generations=G,
                           target_error=0.0)
    h = capi.de_init(cfg)
    try:
        capi.de_run(h)
        x, f = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    assert np.array_equal(x, Xo)
    _, sabs = oracle.evaluate(obj, x, o, M, scale=scale, perm=perm)
    assert np.all(np.abs(f - fo) <= REL64 * (np.abs(fo) + sabs))


def test_batch_with_suite_and_plain_runs_equals_single_runs():
    _need_gpu()
    specs = [(64, 10, 1), (50, 30, 16), (40, 20, 19), (70, 10, 9), (33, 12, 0)]
    cfgs = []
    for r, (np_, d, obj) in enumerate(specs):
        if obj >= 5:
            o, M, perm, scale = _data(obj, d, 30 + r)
        else:
            o, M, perm, scale = problems.shift(d, seed=30 + r), problems.rotation(d, seed=30 + r), None, 1.0
        cfgs.append(capi.make_config(np_, d, objective=obj, shift=o, rot=M, perm=perm, scale=scale, seed=1, run_id=r,
                                     max_generations=20, target_error=0.0))
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
