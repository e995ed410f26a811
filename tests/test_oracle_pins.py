"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself: a
library routine (Triton's Philox4x32-10, numpy's QR, scipy's Rosenbrock),
hand-worked values under tests/golden/, closed forms, exhaustive enumeration,
distributional bounds, and brute-force grid search.  CPU only.
"""
import json
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import problems

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


# ----------------------------------------------------------------------------- Philox
def test_philox_matches_triton_reference():
    """Philox4x32-10 (Salmon et al., SC'11) against Triton's implementation of
    the same published generator, run on the CPU by Triton's interpreter."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(24):
        seed = int(rng.integers(0, 2**63))
        ctr = [int(v) for v in rng.integers(0, 2**32, size=4)]
        cases.append((seed, ctr))
    cases.append((0, [0, 0, 0, 0]))
    cases.append((2**64 - 1, [2**32 - 1] * 4))
    script = textwrap.dedent(
        """
        import os, sys, json
        os.environ["TRITON_INTERPRET"] = "1"
        import torch, triton, triton.language as tl
        @triton.jit
        def k(out, seed, c0, c1, c2, c3):
            a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
            tl.store(out + 0, a); tl.store(out + 1, b); tl.store(out + 2, c); tl.store(out + 3, d)
        res = []
        for seed, ctr in json.loads(sys.stdin.read()):
            o = torch.zeros(4, dtype=torch.int32)
            cs = [torch.tensor(v & 0xFFFFFFFF, dtype=torch.uint32).view(torch.int32).item() for v in ctr]
            sd = seed if seed < 2**63 else seed - 2**64
            k[(1,)](o, sd, *cs)
            res.append([v & 0xFFFFFFFF for v in o.tolist()])
        print(json.dumps(res))
        """
    )
    out = subprocess.run([sys.executable, "-c", script], input=json.dumps(cases), capture_output=True,
                         text=True, timeout=600)
    if out.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + out.stderr[-300:])
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for (seed, ctr), want in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = oracle.philox4x32_10(ctr, key).tolist()
        assert got == want, (seed, ctr)


def test_philox_words_uniform():
    """chi^2 over 256 byte values and per-bit balance over 4096 blocks."""
    words = np.array([oracle.draw(1, 2, 0, 0, g, i, d) for g in range(4) for i in range(32) for d in range(32)],
                     dtype=np.uint64)
    b = np.concatenate([(words >> s) & 0xFF for s in (0, 8, 16, 24)]).astype(np.int64)
    counts = np.bincount(b, minlength=256)
    exp = len(b) / 256.0
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    bits = np.array([[(int(w) >> k) & 1 for k in range(32)] for w in words])
    p = bits.mean(axis=0)
    assert np.all(np.abs(p - 0.5) < 4.5 * math.sqrt(0.25 / len(words)))


def test_draw_counter_layout():
    """Draw d is word d % 4 of block d / 4; the stream fields land in the counter."""
    seed = 0x0123456789ABCDEF
    for (purpose, run_id, cand, g, i, d) in [(1, 0, 0, 0, 0, 0), (2, 3, 5, 7, 11, 13), (2, 1023, 255, 9, 100, 403)]:
        ctr = [d // 4, i, g, (run_id << 12) | (cand << 4) | purpose]
        words = oracle.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.draw(seed, purpose, run_id, cand, g, i, d) == int(words[d % 4])


# ----------------------------------------------------------------------------- maps
def test_u53_closed_forms():
    assert oracle.u53(0, 0) == 0.0
    assert oracle.u53(0x80000000, 0) == 0.5
    assert oracle.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.u53(0, 0x800) == 2.0 ** -53
    assert oracle.u53(0, 0x7FF) == 0.0  # the low 11 bits are dropped


def test_map_index_boundaries():
    """floor(u n / 2^32): the preimage of k is [ceil(k 2^32 / n), ceil((k+1) 2^32 / n))."""
    for n in (1, 2, 3, 7, 10, 100, 1000, 8191, 2**31 + 1):
        for k in {0, 1, n // 2, n - 1}:
            if k >= n:
                continue
            lo = -(-k * 2**32 // n)
            hi = -(-(k + 1) * 2**32 // n) - 1
            assert oracle.map_index(lo, n) == k
            assert oracle.map_index(hi, n) == k
            if lo > 0:
                assert oracle.map_index(lo - 1, n) == k - 1


def test_cr_threshold():
    assert oracle.cr_threshold(0.0) == 0
    assert oracle.cr_threshold(1.0) == 2**32
    assert oracle.cr_threshold(0.5) == 2**31
    assert oracle.cr_threshold(0.9) == math.floor(0.9 * 2**32)


# ----------------------------------------------------------------------------- indices
def test_index_golden_cases():
    g = json.load(open(os.path.join(GOLDEN, "index_draws.json")))
    for c in g["cases"]:
        assert list(oracle.mutant_indices(*c["w"], c["i"], c["np"])) == c["expect"], c["why"]


@pytest.mark.parametrize("np_", [4, 5, 7])
def test_index_triples_exhaustive_bijection(np_):
    """Each (k1, k2, k3) in [0,NP-1) x [0,NP-2) x [0,NP-3) gives a different
    ordered triple of distinct indices != i, so the map covers all of them
    exactly once: uniform draws give the uniform ordered triple (Eq. 2)."""
    def pre(k, n):  # smallest u with floor(u n / 2^32) = k
        return -(-k * 2**32 // n)
    for i in range(np_):
        seen = set()
        for k1 in range(np_ - 1):
            for k2 in range(np_ - 2):
                for k3 in range(np_ - 3):
                    r = oracle.mutant_indices(pre(k1, np_ - 1), pre(k2, np_ - 2), pre(k3, np_ - 3), i, np_)
                    assert len(set(r)) == 3 and i not in r and all(0 <= v < np_ for v in r)
                    seen.add(r)
        n_expected = (np_ - 1) * (np_ - 2) * (np_ - 3)
        assert len(seen) == n_expected


def test_index_triples_chi2_with_philox():
    np_, i = 5, 2
    counts = {}
    n = 0
    for g in range(1, 601):
        for d0 in range(0, 1):
            w = [oracle.draw(7, 2, 0, 0, g, i, k) for k in range(3)]
            r = oracle.mutant_indices(*w, i, np_)
            counts[r] = counts.get(r, 0) + 1
            n += 1
    assert len(counts) == 24
    exp = n / 24.0
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 23 + 6 * math.sqrt(46)


# ----------------------------------------------------------------------------- objectives
def test_objective_golden_values():
    g = json.load(open(os.path.join(GOLDEN, "objective_values.json")))
    for c in g["cases"]:
        f, _ = oracle.objective(c["obj"], np.array(c["x"]))
        assert abs(f - c["f"]) <= g["rtol"] * max(1.0, abs(c["f"])), c


@pytest.mark.parametrize("d", [2, 10, 100])
@pytest.mark.parametrize("obj", [0, 1, 2, 3])
def test_objective_zero_at_shift(obj, d):
    """Sec. 7.3.1: the global minimum 0 sits at the shift vector o."""
    o = problems.shift(d, seed=3)
    M = problems.rotation(d, seed=3)
    f, sabs = oracle.objective(obj, o, o, M)
    if obj == 3:
        assert abs(f) <= 4 * np.finfo(float).eps * (20 + math.e)
    else:
        assert f == 0.0


@pytest.mark.parametrize("obj", [0, 1, 3])
def test_objective_rotation_orientation(obj):
    """x = o + M^T (a e_k) / s gives z = a e_k exactly up to rounding; a
    transposed M would not."""
    d, s = 12, 0.7
    o = problems.shift(d, seed=4)
    M = problems.rotation(d, seed=4)
    for k, a in [(0, 0.5), (5, 2.0), (11, -1.25)]:
        e = np.zeros(d)
        e[k] = a
        x = o + (M.T @ e) / s
        f, _ = oracle.objective(obj, x, o, M, scale=s)
        if obj == 0:
            want = a * a
        elif obj == 1:
            want = a * a - 10 * math.cos(2 * math.pi * a) + 10
        else:
            want = 20 + math.e - 20 * math.exp(-0.2 * math.sqrt(a * a / d)) - math.exp(((d - 1) + math.cos(2 * math.pi * a)) / d)
        assert abs(f - want) <= 1e-11 * (1 + abs(want))
        if obj != 0:  # the sphere is rotation invariant, the others are not
            # the transposed matrix gives a different value (guards the orientation)
            f_t, _ = oracle.objective(obj, x, o, np.ascontiguousarray(M.T), scale=s)
            assert abs(f_t - want) > 1e-6


def test_rosenbrock_matches_scipy():
    """Rosenbrock at t = z + 1 equals scipy.optimize.rosen(t)."""
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(0)
    for d in (2, 3, 10, 50):
        z = rng.uniform(-3, 3, size=d)
        f, _ = oracle.objective(2, z)
        want = float(opt.rosen(z + 1.0))
        assert abs(f - want) <= 1e-13 * abs(want)


def test_rotated_sphere_invariance_and_identity():
    """Orthogonal M leaves the sphere unchanged; M = I equals no rotation."""
    d = 30
    o = problems.shift(d, seed=8)
    M = problems.rotation(d, seed=8)
    X = problems.population(16, d, seed=8)
    f_rot, _ = oracle.evaluate(0, X, o, M)
    f_plain, _ = oracle.evaluate(0, X, o, None)
    assert np.allclose(f_rot, f_plain, rtol=1e-13, atol=0)
    for obj in (0, 1, 2, 3):
        a, _ = oracle.evaluate(obj, X, o, np.eye(d))
        b, _ = oracle.evaluate(obj, X, o, None)
        assert np.array_equal(a, b)


def test_objective_matches_numpy_matmul_rotation():
    """The oracle's scalar rotation loop agrees with numpy's matmul (library
    routine) feeding a sphere, within rounding."""
    d = 50
    o = problems.shift(d, seed=9)
    M = problems.rotation(d, seed=9)
    X = problems.population(8, d, seed=9)
    Z = (X - o) @ M.T
    f, _ = oracle.evaluate(0, X, o, M)
    assert np.allclose(f, (Z * Z).sum(axis=1), rtol=1e-12)


def test_ackley_equal_coordinates():
    for d in (2, 7):
        for a in (1.0, 2.0, 3.0):
            f, _ = oracle.objective(3, np.full(d, a))
            assert abs(f - 20 * (1 - math.exp(-0.2 * a))) <= 1e-13 * 20


# ----------------------------------------------------------------------------- rotation data
@pytest.mark.parametrize("d", [2, 10, 100, 1000])
def test_rotation_orthogonal(d):
    M = problems.rotation(d, seed=1)
    err = np.abs(M.T @ M - np.eye(d)).max()
    assert err <= 1e-12
    g = np.random.default_rng([1, 0, 12]).standard_normal((d, d))
    q, _ = np.linalg.qr(g)
    assert np.allclose(np.abs(M), np.abs(q), atol=1e-12)


# ----------------------------------------------------------------------------- init
def test_init_in_bounds_and_uniform():
    X = oracle.init_population(256, 20, -100.0, 100.0, seed=1)
    assert X.min() >= -100.0 and X.max() < 100.0
    h, _ = np.histogram(X.ravel(), bins=20, range=(-100, 100))
    exp = X.size / 20
    assert ((h - exp) ** 2 / exp).sum() < 19 + 6 * math.sqrt(38)
    assert not np.array_equal(X, oracle.init_population(256, 20, -100.0, 100.0, seed=2))
    assert not np.array_equal(X, oracle.init_population(256, 20, -100.0, 100.0, seed=1, run_id=1))


# ----------------------------------------------------------------------------- one step
def _pop(np_, d, seed, obj=1, rotate=True):
    o = problems.shift(d, seed=seed)
    M = problems.rotation(d, seed=seed) if rotate else None
    X = problems.population(np_, d, seed=seed)
    f, _ = oracle.evaluate(obj, X, o, M)
    return X, f, o, M


def _bits(mask, d):
    return np.array([[(mask[i, j // 32] >> (j % 32)) & 1 for j in range(d)] for i in range(mask.shape[0])],
                    dtype=bool)


def test_step_crossover_properties():
    np_, d = 64, 37
    X, f, o, M = _pop(np_, d, 11)
    for cr in (0.0, 0.3, 0.9, 1.0):
        r = oracle.step(X, f, 0.5, cr, -100, 100, 1, o, M, seed=1, generation=5)
        m = _bits(r["mask"], d)
        assert np.all(m.sum(axis=1) >= 1)
        assert np.all(m[np.arange(np_), r["jrand"]])
        if cr == 0.0:
            assert np.all(m.sum(axis=1) == 1)
        if cr == 1.0:
            assert np.all(m)
        # non-crossed coordinates are the target's own
        assert np.array_equal(r["trial"][~m], X[~m])
    # mean crossed fraction over many generations: CR (D-1)/D + 1/D
    cr = 0.3
    tot = 0
    n = 0
    for g in range(1, 41):
        r = oracle.step(X, f, 0.5, cr, -100, 100, 1, o, M, seed=2, generation=g)
        tot += _bits(r["mask"], d).sum()
        n += np_ * d
    p = cr * (d - 1) / d + 1.0 / d
    sigma = math.sqrt(p * (1 - p) / n)
    assert abs(tot / n - p) < 4 * sigma


def test_step_indices_valid_and_mutation_special_cases():
    np_, d = 50, 9
    X, f, o, M = _pop(np_, d, 12)
    r = oracle.step(X, f, 0.0, 1.0, -100, 100, 0, o, M, seed=3, generation=1)
    idx = r["idx"]
    for i in range(np_):
        assert len(set(idx[i])) == 3 and i not in idx[i] and idx[i].min() >= 0 and idx[i].max() < np_
    # F = 0: the mutant is the base vector x_r1 (no repair is needed inside the box)
    assert np.array_equal(r["trial"], X[idx[:, 0]])
    # F = 1 on a population whose donors differ by exact integers: y = x_r1 + (x_r2 - x_r3)
    Xi = np.tile(np.arange(np_, dtype=float)[:, None], (1, d)) * 0.25
    fi, _ = oracle.evaluate(0, Xi, None, None)
    r = oracle.step(Xi, fi, 1.0, 1.0, -100, 100, 0, None, None, seed=3, generation=2)
    idx = r["idx"]
    want = (idx[:, 0] + idx[:, 1] - idx[:, 2]) * 0.25
    assert np.array_equal(r["trial"], np.tile(want[:, None], (1, d)))


def test_step_repair_keeps_bounds():
    np_, d = 40, 16
    X, f, o, M = _pop(np_, d, 13)
    lo, hi = -100.0, 100.0
    r = oracle.step(X, f, 1.9, 1.0, lo, hi, 1, o, M, seed=4, generation=3)
    t = r["trial"]
    assert t.min() >= lo and t.max() <= hi
    # an out-of-range mutant goes half way from the target to the bound
    idx = r["idx"]
    v = X[idx[:, 0]] + 1.9 * (X[idx[:, 1]] - X[idx[:, 2]])
    low = v < lo
    high = v > hi
    assert low.any() and high.any()
    assert np.allclose(t[low], ((X + lo) * 0.5)[low], rtol=0, atol=0)
    assert np.allclose(t[high], ((X + hi) * 0.5)[high], rtol=0, atol=0)


def test_step_selection():
    np_, d = 64, 10
    X, f, o, M = _pop(np_, d, 14)
    r = oracle.step(X, f, 0.5, 0.9, -100, 100, 1, o, M, seed=5, generation=1)
    acc = r["accept"].astype(bool)
    assert np.array_equal(acc, r["f_trial"] <= f)
    assert np.array_equal(r["X_next"][acc], r["trial"][acc])
    assert np.array_equal(r["X_next"][~acc], X[~acc])
    assert np.all(r["f_next"] <= f)
    fo, _ = oracle.evaluate(1, r["trial"], o, M)
    assert np.array_equal(fo, r["f_trial"])


def test_step_selection_ranks_nan_last():
    """NaN fitness has no quality (Sec. 2, Selection, read with NaN below
    every number): a NaN trial never replaces its target, and every other
    trial, +inf included, replaces a NaN target.  Unrotated Rastrigin with
    o = 0 and scale 1e308 on coordinates in {0, +-100}: y is 0 or +-inf, so f
    is 0 (all coordinates 0) or NaN; +inf comes from scale 1e154."""
    rng = np.random.default_rng(3)
    X = rng.choice([0.0, 100.0, -100.0], size=(64, 2))
    o = np.zeros(2)
    f, _ = oracle.evaluate(1, X, o, None, scale=1e308)
    assert np.isnan(f).any() and (f == 0).any()
    for g in range(1, 6):
        r = oracle.step(X, f, 0.5, 0.9, -100, 100, 1, o, None, seed=7, generation=g, scale=1e308)
        nt, nx = np.isnan(r["f_trial"]), np.isnan(f)
        want = ~nt & (nx | (r["f_trial"] <= f))
        assert np.array_equal(r["accept"].astype(bool), want)
        assert (~nt & nx).any() or g > 1  # the rule that NaN targets are replaced is exercised
        X, f = r["X_next"], r["f_next"]
    # +inf against NaN: with scale 1e154 a coordinate of 100 gives z^2 = 1e312 = +inf
    # and cos(2 pi 1e156) finite, so f = +inf, while the target keeps f = NaN
    Xi = np.full((8, 1), 100.0)
    fi = np.full(8, np.nan)
    r = oracle.step(Xi, fi, 0.5, 0.9, -100, 100, 1, np.zeros(1), None, seed=1, generation=1, scale=1e154)
    assert np.all(np.isposinf(r["f_trial"])) and r["accept"].all()


def test_step_deterministic_and_seeded():
    X, f, o, M = _pop(32, 5, 15)
    a = oracle.step(X, f, 0.5, 0.9, -100, 100, 1, o, M, seed=6, generation=1)
    b = oracle.step(X, f, 0.5, 0.9, -100, 100, 1, o, M, seed=6, generation=1)
    c = oracle.step(X, f, 0.5, 0.9, -100, 100, 1, o, M, seed=6, generation=2)
    assert np.array_equal(a["trial"], b["trial"])
    assert not np.array_equal(a["trial"], c["trial"])


# ----------------------------------------------------------------------------- runs
def test_run_best_non_increasing_and_converges_on_sphere():
    """The small FP64 sphere run (NP=64, D=10, F=0.5, CR=0.9, seed 1) reaches
    the 1e-8 target of Sec. 7.3.4, and greedy selection never raises the best."""
    d = 10
    o = problems.shift(d, seed=1)
    X, f, g, ev, tr = oracle.run(64, d, 0.5, 0.9, -100, 100, 0, o, None, seed=1, max_generations=1000,
                                 target_error=1e-8, trace=True)
    assert np.all(np.diff(tr) <= 0)
    assert f.min() < 1e-8
    assert g < 1000 and ev == 64 * (g + 1)


@pytest.mark.parametrize("obj", [0, 1, 2, 3])
def test_d2_grid_search_agrees_with_de(obj):
    """D = 2: brute force over [-100, 100]^2 (step 0.05) plus local refinement
    finds the same optimum as a DE run."""
    opt = pytest.importorskip("scipy.optimize")
    d = 2
    o = problems.shift(d, seed=21 + obj)
    M = problems.rotation(d, seed=21 + obj)
    xs = np.arange(-100.0, 100.0 + 1e-9, 0.05)
    best_f, best_x = np.inf, None
    for a in range(0, xs.size, 500):
        gx, gy = np.meshgrid(xs[a:a + 500], xs, indexing="ij")
        P = np.stack([gx.ravel(), gy.ravel()], axis=1)
        fv, _ = oracle.evaluate(obj, P, o, M)
        k = int(np.argmin(fv))
        if fv[k] < best_f:
            best_f, best_x = float(fv[k]), P[k].copy()
    res = opt.minimize(lambda x: oracle.objective(obj, x, o, M)[0], best_x, method="Nelder-Mead",
                       options=dict(xatol=1e-12, fatol=1e-20, maxiter=20000))
    x_grid, f_grid = res.x, res.fun
    # DE is a heuristic that can stagnate on a narrow valley (seed 1 does on
    # this Rosenbrock), so the DE optimum is the best of three seeded runs
    runs = [oracle.run(40, d, 0.5, 0.9, -100, 100, obj, o, M, seed=s, max_generations=800, target_error=0.0)
            for s in (1, 2, 3)]
    X, f = min(((r[0], r[1]) for r in runs), key=lambda t: t[1].min())
    b = oracle.best(f)
    assert np.max(np.abs(X[b] - x_grid)) < 1e-6
    assert abs(f[b] - f_grid) < 1e-8
    assert np.max(np.abs(X[b] - o)) < 1e-6


def test_candidate_streams():
    """Candidate stream c of target i uses cand = c in the counter: stream 0 is
    plain DE, other streams give independent trials built the same way."""
    np_, d = 12, 6
    X = problems.population(np_, d, seed=21)
    fX, _ = oracle.evaluate(0, X)
    plain = oracle.step(X, fX, 0.5, 0.9, -100, 100, 0, None, None, seed=3, generation=4)
    zero = oracle.step(X, fX, 0.5, 0.9, -100, 100, 0, None, None, seed=3, generation=4, cand=np.zeros(np_))
    assert np.array_equal(plain["trial"], zero["trial"]) and np.array_equal(plain["idx"], zero["idx"])
    cand = np.arange(np_) % 5
    r = oracle.step(X, fX, 0.5, 0.9, -100, 100, 0, None, None, seed=3, generation=4, cand=cand)
    for i in range(np_):
        w = [oracle.draw(3, oracle.PURPOSE_STEP, 0, int(cand[i]), 4, i, k) for k in range(4)]
        assert tuple(r["idx"][i]) == oracle.mutant_indices(w[0], w[1], w[2], i, np_)
        assert r["jrand"][i] == oracle.map_index(w[3], d)
    differ = [i for i in range(np_) if cand[i] != 0]
    assert any(not np.array_equal(r["idx"][i], plain["idx"][i]) for i in differ)
