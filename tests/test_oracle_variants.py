"""Pins of the oracle's DE variants (Sec. 2 names them: base "best", "exp"
crossover, jDE's per-individual F and CR) against special cases, structural
facts and the published distributions.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import problems


def _fma(a, b, c):
    """a * b + c with one rounding (exact rational arithmetic, then the
    correctly rounded conversion to float)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _bits(mask, d):
    return np.array([[(int(mask[i, j // 32]) >> (j % 32)) & 1 for j in range(d)] for i in range(mask.shape[0])],
                    dtype=bool)


def test_best1bin_with_zero_weight_copies_the_best():
    np_, d = 40, 7
    X = problems.population(np_, d, seed=1)
    fX, _ = oracle.evaluate(0, X)
    fX[5] = fX[9] = fX.min() - 1.0  # a tie for the best: the lower index wins
    r = oracle.step(X, fX, 0.0, 1.0, -100, 100, 0, None, None, seed=2, generation=3, strategy=1)
    assert np.all(r["trial"] == X[5])


def test_best1bin_differences_use_the_first_two_donors():
    np_, d = 30, 5
    X = problems.population(np_, d, seed=3)
    fX, _ = oracle.evaluate(0, X)
    b = int(np.argmin(fX))
    r = oracle.step(X, fX, 0.5, 1.0, -1e9, 1e9, 0, None, None, seed=4, generation=2, strategy=1)
    for i in range(np_):
        r1, r2, _ = r["idx"][i]
        expect = np.array([_fma(0.5, X[r1, j] - X[r2, j], X[b, j]) for j in range(d)])
        assert np.array_equal(r["trial"][i], expect)


def test_exp_crossover_is_one_cyclic_block_from_the_start():
    np_, d = 300, 9
    X = problems.population(np_, d, seed=5)
    fX, _ = oracle.evaluate(0, X)
    r = oracle.step(X, fX, 0.5, 0.6, -100, 100, 0, None, None, seed=6, generation=1, strategy=2)
    m = _bits(r["mask"], d)
    for i in range(np_):
        n = r["jrand"][i]
        L = int(m[i].sum())
        assert 1 <= L <= d and m[i, n]
        assert all(m[i, (n + k) % d] for k in range(L))


@pytest.mark.parametrize("cr,expect_all", [(0.0, False), (1.0, True)])
def test_exp_crossover_extremes(cr, expect_all):
    np_, d = 50, 6
    X = problems.population(np_, d, seed=7)
    fX, _ = oracle.evaluate(0, X)
    r = oracle.step(X, fX, 0.5, cr, -100, 100, 0, None, None, seed=8, generation=1, strategy=2)
    m = _bits(r["mask"], d)
    if expect_all:
        assert m.all()
    else:
        assert np.all(m.sum(axis=1) == 1) and np.all(m[np.arange(np_), r["jrand"]])


def test_exp_crossover_length_follows_the_truncated_geometric_law():
    np_, d, cr = 4000, 10, 0.7
    X = problems.population(np_, d, seed=9)
    fX, _ = oracle.evaluate(0, X)
    r = oracle.step(X, fX, 0.5, cr, -100, 100, 0, None, None, seed=10, generation=1, strategy=2)
    L = _bits(r["mask"], d).sum(axis=1)
    # P(L = l) = cr^(l-1) (1 - cr) for l < d, P(L = d) = cr^(d-1)
    p = np.array([cr ** (l - 1) * (1 - cr) for l in range(1, d)] + [cr ** (d - 1)])
    mean = float(np.dot(np.arange(1, d + 1), p))
    var = float(np.dot((np.arange(1, d + 1) - mean) ** 2, p))
    assert mean == pytest.approx((1 - cr ** d) / (1 - cr), rel=1e-12)
    assert abs(L.mean() - mean) < 4 * math.sqrt(var / np_)
    counts = np.bincount(L, minlength=d + 1)[1:]
    chi2 = float(np.sum((counts - np_ * p) ** 2 / (np_ * p)))
    assert chi2 < 30.0  # 9 degrees of freedom


def test_jde_parameters_adapt_at_the_published_rate():
    np_, d = 4000, 5
    X = problems.population(np_, d, seed=11)
    fX, _ = oracle.evaluate(0, X)
    r = oracle.step(X, fX, 0.5, 0.9, -100, 100, 0, None, None, seed=12, generation=1, jde=True)
    F1, C1 = r["F_next"], r["CR_next"]
    acc = r["accept"].astype(bool)
    # rejected trials keep the old parameters
    assert np.all(F1[~acc] == 0.5) and np.all(C1[~acc] == 0.9)
    # new values lie in the published ranges
    assert np.all((F1 >= 0.1) & (F1 <= 1.0)) and np.all((C1 >= 0.0) & (C1 < 1.0))
    # each parameter changes with probability 0.1 (independently of acceptance)
    n = acc.sum()
    for changed in (F1[acc] != 0.5, C1[acc] != 0.9):
        k = changed.sum()
        assert abs(k - 0.1 * n) < 4 * math.sqrt(0.1 * 0.9 * n), (k, n)


def test_jde_carries_parameters_across_generations():
    np_, d = 64, 6
    o = problems.shift(d, seed=13)
    X, f, g, ev, _, jF, jCR = oracle.run(np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=13, max_generations=30,
                                         target_error=0.0, jde=True, return_adaptive=True)
    assert g == 30
    assert np.all((jF >= 0.1) & (jF <= 1.0)) and np.all((jCR >= 0.0) & (jCR <= 1.0))
    assert np.any(jF != 0.5) and np.any(jCR != 0.9)


@pytest.mark.parametrize("strategy,jde", [(2, False), (0, True), (1, True)])
def test_variants_solve_the_small_sphere(strategy, jde):
    d = 10
    o = problems.shift(d, seed=1)
    X, f, g, ev, _ = oracle.run(64, d, 0.5, 0.9, -100, 100, 0, o, None, seed=1, max_generations=3000,
                                target_error=1e-8, strategy=strategy, jde=jde)
    assert f.min() < 1e-8 and g < 3000


def test_best1bin_converges_then_stalls_on_a_collapsed_population():
    """DE/best/1 with fixed F = 0.5 pulls every trial towards the best and
    can collapse the population (all rows equal, zero differences): the
    sphere improves by many orders of magnitude, then the run stalls."""
    d = 10
    o = problems.shift(d, seed=1)
    X, f, g, ev, tr = oracle.run(64, d, 0.5, 0.9, -100, 100, 0, o, None, seed=1, max_generations=3000,
                                 target_error=1e-8, strategy=1, trace=True)
    assert tr[-1] < 1e-2 * tr[0]
    if f.min() >= 1e-8:  # stalled: the population has collapsed onto one point
        assert np.all(np.ptp(X, axis=0) == 0.0)
