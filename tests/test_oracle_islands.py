"""Pins of the oracle's island model (Sec. 3.2, Sec. 5.4): independent islands
are single runs, one migration step moves the ring's best into the worst
slots, and the model stops with its first island to reach the target; with
asynchronous migration the islands are single runs until the second
migration point, where the migrants are the predecessor's best of the first.
CPU only."""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import problems


def test_ranked_selection_order_ties_and_nan():
    f = np.array([3.0, 1.0, np.nan, 1.0, 5.0, 5.0, 0.5])
    assert list(oracle.island_ranked(f, 4)) == [6, 1, 3, 0]
    assert list(oracle.island_ranked(f, 4, worst=True)) == [2, 5, 4, 0]


def test_islands_without_migration_are_single_runs():
    m, np_, d, G = 3, 24, 6, 30
    o = problems.shift(d, seed=2)
    X, f, g, ev, _, _ = oracle.run_islands(m, 0, 1, np_, d, 0.5, 0.9, -100, 100, 1, o, None, seed=4,
                                           max_generations=G, target_error=0.0, run_id=7)
    assert g == G and ev == np_ * (1 + G)
    for k in range(m):
        Xs, fs, gs, _, _ = oracle.run(np_, d, 0.5, 0.9, -100, 100, 1, o, None, seed=4, max_generations=G,
                                      target_error=0.0, run_id=7 + k)
        assert np.array_equal(X[k], Xs) and np.array_equal(f[k], fs)


@pytest.mark.parametrize("nmig", [1, 3])
def test_one_migration_moves_the_best_into_the_next_islands_worst(nmig):
    m, np_, d = 4, 20, 5
    o = problems.shift(d, seed=3)
    X0, f0, _, _, _, _ = oracle.run_islands(m, 0, nmig, np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=5,
                                            max_generations=1, target_error=0.0)
    X1, f1, _, _, _, _ = oracle.run_islands(m, 1, nmig, np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=5,
                                            max_generations=1, target_error=0.0)
    for k in range(m):
        src, dst = k, (k + 1) % m
        best = np.lexsort((np.arange(np_), f0[src]))[:nmig]
        worst = np.lexsort((-np.arange(np_), -f0[dst]))[:nmig]
        Xw, fw = X0[dst].copy(), f0[dst].copy()
        Xw[worst] = X0[src][best]
        fw[worst] = f0[src][best]
        assert np.array_equal(X1[dst], Xw) and np.array_equal(f1[dst], fw)


def test_jde_migrants_carry_their_parameters():
    m, np_, d = 3, 16, 4
    o = problems.shift(d, seed=6)
    X0, f0, _, _, F0, C0 = oracle.run_islands(m, 0, 2, np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=8,
                                              max_generations=3, target_error=0.0, jde=True)
    X1, f1, _, _, F1, C1 = oracle.run_islands(m, 3, 2, np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=8,
                                              max_generations=3, target_error=0.0, jde=True)
    for k in range(m):
        src, dst = k, (k + 1) % m
        best = oracle.island_ranked(f0[src], 2)
        worst = oracle.island_ranked(f0[dst], 2, worst=True)
        assert np.array_equal(F1[dst][worst], F0[src][best]) and np.array_equal(C1[dst][worst], C0[src][best])


def test_the_model_stops_with_its_first_island_to_reach_the_target():
    m, np_, d = 4, 32, 5
    o = problems.shift(d, seed=9)
    gs = [oracle.run(np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=10, max_generations=2000, target_error=1e-8,
                     run_id=k)[2] for k in range(m)]
    X, f, g, ev, _, _ = oracle.run_islands(m, 0, 1, np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=10,
                                           max_generations=2000, target_error=1e-8)
    assert g == min(gs)
    assert f.min() < 1e-8


def test_migration_keeps_the_model_best_non_increasing():
    m, np_, d = 4, 20, 10
    o, M = problems.shift(d, seed=11), problems.rotation(d, seed=11)
    prev = np.inf
    for G in range(0, 60, 6):
        _, f, _, _, _, _ = oracle.run_islands(m, 5, 2, np_, d, 0.5, 0.9, -100, 100, 1, o, M, seed=12,
                                              max_generations=G, target_error=0.0)
        assert f.min() <= prev
        prev = f.min()


# ----------------------------------------------------------------- asynchronous
def _plain(np_, d, obj, o, M, seed, G, run_id):
    """One island's single run (no migration) after G generations."""
    X, f, _, _, _ = oracle.run(np_, d, 0.5, 0.9, -100, 100, obj, o, M, seed=seed, max_generations=G,
                               target_error=0.0, run_id=run_id)
    return X, f


@pytest.mark.parametrize("G", [4, 5, 9])
def test_async_islands_are_single_runs_before_the_second_migration_point(G):
    """Interval 5: the first migration point (generation 5) only posts, so up
    to generation 9 every island is its own single run."""
    m, np_, d, obj = 3, 20, 6, 1
    o = problems.shift(d, seed=21)
    X, f, g, _, _, _ = oracle.run_islands(m, 5, 2, np_, d, 0.5, 0.9, -100, 100, obj, o, None, seed=22,
                                          max_generations=G, target_error=0.0, run_id=3, asynchronous=True)
    assert g == G
    for k in range(m):
        Xs, fs = _plain(np_, d, obj, o, None, 22, G, 3 + k)
        assert np.array_equal(X[k], Xs) and np.array_equal(f[k], fs)


@pytest.mark.parametrize("nmig", [1, 3])
def test_async_migrants_are_the_predecessors_best_one_interval_earlier(nmig):
    """At the second migration point (generation 10, interval 5) island k's
    nmig worst (of its own single run after 10 generations) hold the nmig best
    of island k - 1's single run after 5 generations, the q-th best in the
    q-th worst, with their fitness."""
    m, np_, d, obj, I = 4, 24, 5, 3, 5
    o, M = problems.shift(d, seed=23), problems.rotation(d, seed=23)
    X, f, _, _, _, _ = oracle.run_islands(m, I, nmig, np_, d, 0.5, 0.9, -100, 100, obj, o, M, seed=24,
                                          max_generations=2 * I, target_error=0.0, asynchronous=True)
    early = [_plain(np_, d, obj, o, M, 24, I, k) for k in range(m)]
    late = [_plain(np_, d, obj, o, M, 24, 2 * I, k) for k in range(m)]
    for k in range(m):
        src = (k - 1) % m
        best = np.lexsort((np.arange(np_), early[src][1]))[:nmig]
        worst = np.lexsort((-np.arange(np_), -late[k][1]))[:nmig]
        Xw, fw = late[k][0].copy(), late[k][1].copy()
        Xw[worst] = early[src][0][best]
        fw[worst] = early[src][1][best]
        assert np.array_equal(X[k], Xw) and np.array_equal(f[k], fw)


def test_async_jde_migrants_carry_their_parameters_from_the_previous_point():
    m, np_, d, I = 3, 16, 4, 3
    o = problems.shift(d, seed=25)
    X, f, _, _, F, C = oracle.run_islands(m, I, 2, np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=26,
                                          max_generations=2 * I, target_error=0.0, jde=True, asynchronous=True)
    Xe, fe, _, _, Fe, Ce = oracle.run_islands(m, 0, 2, np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=26,
                                              max_generations=I, target_error=0.0, jde=True)
    Xl, fl, _, _, Fl, Cl = oracle.run_islands(m, 0, 2, np_, d, 0.5, 0.9, -100, 100, 0, o, None, seed=26,
                                              max_generations=2 * I, target_error=0.0, jde=True)
    for k in range(m):
        src = (k - 1) % m
        best = oracle.island_ranked(fe[src], 2)
        worst = oracle.island_ranked(fl[k], 2, worst=True)
        assert np.array_equal(F[k][worst], Fe[src][best]) and np.array_equal(C[k][worst], Ce[src][best])
        keep = np.setdiff1d(np.arange(np_), worst)
        assert np.array_equal(F[k][keep], Fl[k][keep]) and np.array_equal(X[k][keep], Xl[k][keep])


def test_async_and_sync_migration_differ_and_keep_the_best_non_increasing():
    m, np_, d = 4, 20, 10
    o, M = problems.shift(d, seed=27), problems.rotation(d, seed=27)
    fa = oracle.run_islands(m, 4, 2, np_, d, 0.5, 0.9, -100, 100, 1, o, M, seed=28, max_generations=24,
                            target_error=0.0, asynchronous=True)[1]
    fs = oracle.run_islands(m, 4, 2, np_, d, 0.5, 0.9, -100, 100, 1, o, M, seed=28, max_generations=24,
                            target_error=0.0)[1]
    assert not np.array_equal(fa, fs)
    prev = np.inf
    for G in range(0, 40, 4):
        f = oracle.run_islands(m, 4, 2, np_, d, 0.5, 0.9, -100, 100, 1, o, M, seed=28, max_generations=G,
                               target_error=0.0, asynchronous=True)[1]
        assert f.min() <= prev
        prev = f.min()
