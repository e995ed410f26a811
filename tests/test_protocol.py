"""The benchmark protocol's scoring (Sec. 7.3.5): rank-sum with averaged
ties and the n (n + 1) / 2 correction.  Host logic, CPU only."""
import itertools
import random

import pytest

from paper_2405_16551_gb300.protocol import Trial, benchmark_scores, final_ranking, function_scores


def T(err, sec=1.0):
    return Trial(error=err, seconds=sec, evals=0, generations=0)


def test_dominating_algorithm_takes_the_top_ranks():
    s = function_scores({"A": [T(1e-3), T(1e-4), T(1e-5)], "B": [T(1.0), T(2.0), T(3.0)]})
    # A holds ranks 4, 5, 6; B ranks 1, 2, 3; correction 3 * 4 / 2 = 6
    assert s == {"A": 9.0, "B": 0.0}


def test_solved_trials_beat_unsolved_ones_and_order_by_time():
    s = function_scores({"fast": [T(1e-9, 2.0), T(5.0, 1.0)], "slow": [T(1e-10, 3.0), T(4.0, 0.1)]})
    # order worst -> best: 5.0 (fast), 4.0 (slow), solved in 3 s (slow), solved in 2 s (fast)
    assert s == {"fast": 1 + 4 - 3, "slow": 2 + 3 - 3}


def test_ties_share_the_average_rank():
    s = function_scores({"A": [T(0.5), T(0.25)], "B": [T(0.5), T(1.0)]})
    # worst -> best: 1.0 (B, rank 1), 0.5 (A, B: ranks 2 and 3 -> 2.5 each), 0.25 (A, rank 4)
    assert s == {"A": 2.5 + 4 - 3, "B": 1 + 2.5 - 3}


def test_scores_sum_to_the_rank_total_minus_the_corrections():
    rng = random.Random(5)
    for n, m in itertools.product([1, 3, 30], [1, 2, 5]):
        trials = {f"a{j}": [T(rng.choice([1e-9, 1e-3, 0.5, 2.0]), rng.choice([1.0, 2.0])) for _ in range(n)]
                  for j in range(m)}
        s = function_scores(trials)
        N = n * m
        assert sum(s.values()) == pytest.approx(N * (N + 1) / 2 - m * n * (n + 1) / 2)
        for v in s.values():
            assert 0 <= v <= n * N - n * (n + 1) / 2 + 1e-9


def test_benchmark_score_and_final_ranking():
    per_fn = {
        "F1": {"A": [T(1e-3)], "B": [T(1.0)], "C": [T(1e-3)]},
        "F2": {"A": [T(2.0)], "B": [T(1.0)], "C": [T(3.0)]},
    }
    tot = benchmark_scores(per_fn)
    # F1: B rank 1, A and C 2.5 each; F2: C 1, A 2, B 3; correction 1 per function
    assert tot == {"A": 1.5 + 1, "B": 0 + 2, "C": 1.5 + 0}
    assert final_ranking(tot) == {"A": 1, "B": 2, "C": 3}
    assert final_ranking({"x": 1.0, "y": 1.0, "z": 0.0}) == {"x": 1, "y": 1, "z": 3}


def test_unequal_trial_counts_are_rejected():
    with pytest.raises(ValueError):
        function_scores({"A": [T(1.0)], "B": [T(1.0), T(2.0)]})
