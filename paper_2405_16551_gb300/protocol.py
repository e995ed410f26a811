"""The benchmark protocol the paper proposes for GPU DEs (Sec. 7.3.4 stopping
criteria, Sec. 7.3.5 evaluation criteria).

* A trial stops when its error (best f; every function of the suite has
  f* = 0) falls below 1e-8, or when the evaluation budget (5e6 for D = 50,
  1e7 for D = 100) is spent.  Each trial records its minimum error, its
  wall-clock time and the evaluations it used.
* Scoring: for one function, all trials of all m algorithms (n trials each)
  are ranked together from worst (rank 1) to best (rank n m); tied trials
  share the average of their ranks.  A trial that reached the target beats
  one that did not; two that reached it are ordered by wall-clock time, two
  that did not by their error.  An algorithm's score is the sum of its
  trials' ranks minus n (n + 1) / 2; the benchmark score is the sum over
  functions.

Trials run as one batched handle per (algorithm, function): every trial is
one run of the batch, all of them advance in lockstep, and a trial's
wall-clock time is the batch time up to the generation at which it stopped
(batch seconds x its generations / the batch's generations).

This module is host logic over the C ABI (``capi``); it computes no step of
the DE method itself.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

TARGET = 1e-8
BUDGET = {50: 5_000_000, 100: 10_000_000}


@dataclass
class Trial:
    error: float
    seconds: float
    evals: int
    generations: int


@dataclass
class Algorithm:
    """One competing configuration: fixed parameters for every function
    (Sec. 7.3.4 forbids tuning per problem or dimension)."""
    name: str
    np_: int
    f: float = 0.5
    cr: float = 0.9
    strategy: int = 0
    jde: bool = False
    precision: int = 0
    extra: dict = field(default_factory=dict)


def _key(t: Trial, target: float = TARGET):
    """Smaller is better: solved trials by time, then unsolved ones by error."""
    if t.error < target:
        return (0, t.seconds)
    return (1, t.error if np.isfinite(t.error) else np.inf)


def function_scores(trials: dict, target: float = TARGET) -> dict:
    """Scores of the algorithms on one function.  trials: name -> list of n
    Trial (the same n for every algorithm)."""
    names = list(trials)
    n = len(trials[names[0]])
    if any(len(trials[a]) != n for a in names):
        raise ValueError("every algorithm needs the same number of trials")
    flat = [(_key(t, target), a) for a in names for t in trials[a]]
    N = len(flat)
    # worst first: rank 1 .. N, ties take the average rank
    order = sorted(range(N), key=lambda k: flat[k][0], reverse=True)
    ranks = [0.0] * N
    pos = 0
    while pos < N:
        end = pos
        while end + 1 < N and flat[order[end + 1]][0] == flat[order[pos]][0]:
            end += 1
        avg = (pos + 1 + end + 1) / 2.0
        for q in range(pos, end + 1):
            ranks[order[q]] = avg
        pos = end + 1
    score = {a: 0.0 for a in names}
    for k, (_, a) in enumerate(flat):
        score[a] += ranks[k]
    corr = n * (n + 1) / 2.0
    return {a: score[a] - corr for a in names}


def benchmark_scores(per_function: dict, target: float = TARGET) -> dict:
    """Sum of the function scores; per_function: function -> (name -> trials)."""
    total: dict = {}
    for trials in per_function.values():
        for a, s in function_scores(trials, target).items():
            total[a] = total.get(a, 0.0) + s
    return total


def final_ranking(total: dict) -> dict:
    """1 for the highest benchmark score (the best), ties share the better place."""
    order = sorted(total, key=lambda a: -total[a])
    rank, out = 0, {}
    for k, a in enumerate(order):
        if k == 0 or total[a] != total[order[k - 1]]:
            rank = k + 1
        out[a] = rank
    return out


def run_trials(capi, alg: Algorithm, objective: int, d: int, data: dict, ntrials: int, budget: int,
               seed: int = 1, stream=None, synchronize=None) -> list:
    """ntrials trials of one algorithm on one function as one batched handle
    (run_id = trial index); returns a Trial per trial."""
    cfgs = []
    for t in range(ntrials):
        cfgs.append(capi.make_config(alg.np_, d, f=alg.f, cr=alg.cr, objective=objective, shift=data["shift"],
                                     rot=data["rot"], perm=data.get("perm"), scale=data.get("scale", 1.0),
                                     seed=seed, run_id=t, precision=alg.precision, target_error=TARGET,
                                     max_evals=budget, max_generations=budget // alg.np_ + 1,
                                     strategy=alg.strategy, jde=alg.jde, **alg.extra))
    h = capi.de_init_batch(cfgs, stream=stream)
    try:
        if synchronize:
            synchronize()
        t0 = time.perf_counter()
        res = capi.de_run(h, ntrials)
        secs = time.perf_counter() - t0
    finally:
        capi.de_destroy(h)
    gmax = max(r["generations"] for r in res) or 1
    return [Trial(error=float(r["best_f"]), seconds=secs * r["generations"] / gmax, evals=int(r["evals"]),
                  generations=int(r["generations"])) for r in res]
