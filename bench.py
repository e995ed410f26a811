"""Throughput of the DE/rand/1/bin generation step on GB300.

Workload (the rotated-shifted Rastrigin configuration): NP = 1024, D = 100,
F = 0.5, CR = 0.9, bounds [-100, 100]^D, shift o ~ U[-80, 80]^D, M orthogonal
from the QR of a seeded Gaussian, 3000 generations.  One "step" is one whole
run of that workload: initialise + evaluate the population, then 3000
generations of mutation, crossover, repair, rotation + objective and
selection, with the best-so-far record and stop test after each generation.

Metric: trial evaluations per second (NP x generations per run / time).

* value          device time (CUDA events on the library's stream) summed
                 over the K timed runs; inputs resident in HBM; L2 flushed
                 (a 512 MiB write) between runs.
* e2e            the same runs through the C ABI with host inputs: de_init
                 from pinned host shift/rotation, de_run, de_get_best back to
                 host, de_destroy, wall clock.
* roofline       the dominant kernel's algorithmic work per launch over its
                 average launch time (events around the generations only).
* cpu_baseline   the FP64 CPU oracle on a bounded sample of the same
                 workload, timed on this host's cores.

``--impl reference`` times the oracle itself as the reference arm.
Multi-GPU (torchrun): every rank runs its own independent replica of the
workload (run_id = rank), no collective on the data path ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NP, D, F, CR, GENS, SEED = 1024, 100, 0.5, 0.9, 3000, 1
OBJ_RASTRIGIN = 1
WORKLOAD = "rotated-shifted Rastrigin NP=1024 D=100 F=0.5 CR=0.9 3000 generations"
METRIC = "trial evals/sec (DE/rand/1/bin, D=100, NP=1024, rotated-shifted Rastrigin)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--precision", default="auto", choices=["auto", "fp64", "bf16x3", "tf32x3"])
    p.add_argument("--generations", type=int, default=GENS)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the other precision forms")
    p.add_argument("--workload", default="rastrigin",
                   choices=["rastrigin", "sphere_small", "batch512", "ode_surrogate", "stress", "stress_batch",
                            "variants", "suite", "islands", "accuracy", "split_error"],
                   help="rastrigin: the headline configuration (default); the others measure the batched, "
                        "surrogate and large-dimension configurations with the same harness")
    return p.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if "Active" in s[4 + k] and "Not" not in s[4 + k]:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ----------------------------------------------------------------------------- problem
def make_problem():
    from paper_2405_16551_gb300 import problems

    return problems.shift(D, seed=SEED), problems.rotation(D, seed=SEED)


def cpu_baseline(o, M, budget_s=12.0):
    """The FP64 oracle, as it stands, on all host cores (the paper's
    master-slave form: evaluations spread over a thread pool), on a bounded
    sample: a first run of a few generations sizes a second run to about
    budget_s seconds of CPU time."""
    import oracle

    cores = os.cpu_count() or 1
    oracle.build()

    def timed(gens):
        t0 = time.perf_counter()
        _, _, g, ev, _ = oracle.run(NP, D, F, CR, -100.0, 100.0, OBJ_RASTRIGIN, o, M, seed=SEED,
                                    max_generations=gens, target_error=1e-8, threads=cores)
        return g, ev, time.perf_counter() - t0

    g0, _, t0 = timed(4)
    per_gen = max(t0 / max(g0 + 1, 1), 1e-4)
    gens = int(min(GENS, max(4, budget_s / per_gen)))
    g, ev, dt = timed(gens)
    # every evaluation the timed call made counts: the initial population's
    # NP and NP per generation (FE = NP (1 + g))
    return {"value": ev / dt, "unit": "trial evals/s", "cores": cores, "kind": "oracle",
            "sample": f"init + {g} of the {GENS} generations of the same workload (NP={NP}, D={D}), FP64, "
                      f"OpenMP over individuals for evaluation; {ev} evaluations counted (NP x (1 + {g})); "
                      f"{dt:.2f} s"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    o, M = make_problem()
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    sample_gens = 4
    times, evals = [], 0
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, _, _, ev, _ = oracle.run(NP, D, F, CR, -100.0, 100.0, OBJ_RASTRIGIN, o, M, seed=SEED,
                                    max_generations=sample_gens, target_error=1e-8, threads=cores)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
            evals += ev
    tot = sum(times)
    # every evaluation of a timed step counts: the initial population's NP
    # and NP per generation, NP (1 + sample_gens) per step
    value = evals / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "trial evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"init + {sample_gens} generations (bounded CPU sample)",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "trial evals/s", "cores": cores, "kind": "oracle",
                             "sample": f"init + {sample_gens} generations per step, NP x (1 + {sample_gens}) "
                                       "evaluations counted per step, FP64, OpenMP over individuals"},
            "e2e": {"value": value, "unit": "trial evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- gb300 arm
PREC_NAMES = {"fp64": 0, "bf16x3": 1, "tf32x3": 2}
DTYPE = {"fp64": "f64", "bf16x3": "bf16x3 products, f32 accumulate, f64 trials and selection band",
         "tf32x3": "tf32x3 products, f32 accumulate, f64 trials and selection band"}


# de_get_plan's kernel paths
KERNEL_PATH_NAMES = {0: "fp64 fused", 1: "split three-kernel", 2: "split persistent cluster",
                     3: "fp64 cooperative persistent", 4: "split persistent, CTA-local products (cooperative)",
                     5: "split persistent batch, per-run arrival counters (cooperative)"}


def launches_per_step(plan, G):
    """Kernels one timed step launches: re-initialisation (population,
    evaluation, best record) plus the generations."""
    path = plan["kernel_path"]
    if path == 0:
        return 3 + G          # one fused FP64 kernel per generation
    if path == 1:
        return 3 + 3 * G      # trial, tensor-core fitness, FP64 band per generation
    if path == 3:
        return 3 + 1          # one cooperative FP64 kernel for all generations
    if path == 5:
        return 3 + 1          # one persistent batch kernel for all generations
    return 3 + 2              # one persistent split kernel (path 2 or 4) for all generations, then its close-out


def measure(capi, torch, prec_name, G, steps, warmup, rank, flush, stream):
    """Device-timed steps of one precision form: events around re-initialisation
    + G generations; L2 flushed between steps outside the events."""
    o, M = make_problem()
    from paper_2405_16551_gb300 import replicas

    cfg = capi.make_config(NP, D, f=F, cr=CR, objective=OBJ_RASTRIGIN, shift=o, rot=M, seed=SEED,
                           run_id=replicas.replica_run_id(0, rank),
                           precision=PREC_NAMES[prec_name], target_error=1e-8, max_generations=G)
    h = capi.de_init(cfg, stream=stream.cuda_stream)
    plan = capi.de_get_plan(h)

    def one_step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        capi.de_reset(h)
        if evs is not None:
            evs[1].record(stream)
        capi.de_step(h, G)
        if evs is not None:
            evs[2].record(stream)

    for _ in range(warmup):
        one_step()
        flush.zero_()
    torch.cuda.synchronize()
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for k in range(steps):
        one_step(events[k])
        flush.zero_()
    torch.cuda.synchronize()
    step_ms = [e[0].elapsed_time(e[2]) for e in events]
    gen_ms = [e[1].elapsed_time(e[2]) for e in events]
    best = capi.de_get_best(h)
    stats = capi.de_get_stats(h)
    capi.de_destroy(h)
    return dict(dev_ms=sum(step_ms), gen_ms=sum(gen_ms), plan=plan, best_f=best["best_f"], stats=stats)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    from paper_2405_16551_gb300 import capi, replicas

    torch.cuda.set_device(local)
    if args.workload != "rastrigin":
        line = run_workload(args, capi, torch, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    prec_name = args.precision if args.precision != "auto" else os.environ.get("DE_BENCH_PRECISION", "bf16x3")
    G = args.generations
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    head = measure(capi, torch, prec_name, G, args.steps, args.warmup, rank, flush, stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    dev_ms, gen_ms = replicas.max_over_ranks([head["dev_ms"], head["gen_ms"]], dist, device="cuda")
    trials_per_step = NP * G
    value = replicas.job_rate(trials_per_step * args.steps, world, dev_ms / 1e3)

    # the other precision forms on the same device, for the comparison with
    # the plain FP64 GPU DE (two steps each)
    forms = {}
    if not args.no_forms:
        for name in ("fp64", "bf16x3", "tf32x3"):
            if name == prec_name:
                r = head
                k = args.steps
            else:
                r = measure(capi, torch, name, G, 2, 1, rank, flush, stream)
                k = 2
            forms[name] = {"trial_evals_per_s": trials_per_step * k / (r["dev_ms"] / 1e3),
                           "us_per_generation": 1e3 * r["gen_ms"] / (k * G), "kernel_path": r["plan"]["kernel_path"],
                           "best_f": r["best_f"], "fp64_reevaluations": r["stats"]["fp64_reevals"]}
        base = forms["fp64"]["trial_evals_per_s"]
        for name in forms:
            forms[name]["speedup_vs_fp64_gpu"] = forms[name]["trial_evals_per_s"] / base

    # e2e through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        o, M = make_problem()
        o_pin = torch.from_numpy(o).pin_memory()
        m_pin = torch.from_numpy(np.ascontiguousarray(M)).pin_memory()
        cfg_e = capi.make_config(NP, D, f=F, cr=CR, objective=OBJ_RASTRIGIN, shift=o_pin.numpy(), rot=m_pin.numpy(),
                                 seed=SEED, run_id=replicas.replica_run_id(0, rank),
                                 precision=PREC_NAMES[prec_name], target_error=1e-8,
                                 max_generations=G)
        times = []
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            he = capi.de_init(cfg_e, stream=stream.cuda_stream)
            capi.de_run(he)
            capi.de_get_best(he)
            capi.de_destroy(he)
            torch.cuda.synchronize()
            if k >= args.warmup:
                times.append(time.perf_counter() - t0)
            flush.zero_()
        tot = replicas.max_over_ranks([sum(times)], dist, device="cuda")[0]
        e2e = {"value": replicas.job_rate(trials_per_step * args.steps, world, tot), "unit": "trial evals/s",
               "h2d_bytes_per_step": 8 * (D + D * D), "d2h_bytes_per_step": 8 * (D + 1) + 48}

    # the device's measured FP64 rate (DFMA chains on every SM), the peak of
    # the FP64 kernels
    fp64_peak = capi.de_selftest_fp64_rate()
    if forms:
        f64 = forms["fp64"]
        f64["fp64_tflops"] = NP * (2.0 * D * D + 9.0 * D) / (f64["us_per_generation"] * 1e-6) / 1e12
        f64["fp64_frac_of_measured_rate"] = f64["fp64_tflops"] / fp64_peak

    clk = clocks.stop()

    # roofline of the dominant kernel
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    path = head["plan"]["kernel_path"]
    avg_gen_us = 1e3 * gen_ms / (args.steps * G)
    if path in (0, 3):
        flops = NP * (2.0 * D * D + 9.0 * D)
        achieved = flops / (avg_gen_us * 1e-6) / 1e12
        roof = {"bound": "alu", "kernel": "k_gen_fp64" if path == 0 else "k_gen_fp64_persist",
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": None,
                "peak_source": "de_selftest_fp64_rate: independent DFMA chains on every SM of this device, "
                               "measured in this run (of measured)"}
    else:
        # algorithmic bytes per trial: read the target row, write the next
        # generation's row, fitness in and out
        byts = NP * (2 * 8 * D + 16)
        persistent = path in (2, 4)
        kname = {2: "k_persist", 4: "k_persist_cta"}.get(path, "k_trial_split + k_fit_tc + k_band_fp64")
        per_launch = byts * G if persistent else byts
        launch_us = avg_gen_us * G if persistent else avg_gen_us
        achieved = per_launch / (launch_us * 1e-6) / 1e9
        pk = float(peaks.get("hbm_gbs", 6800.0))
        roof = {"bound": "hbm", "kernel": kname,
                "achieved": achieved, "peak": pk, "unit": "GB/s", "frac": achieved / pk,
                "traffic": TRAFFIC_PER_LAUNCH.get((kname, G)) if persistent else None,
                "algorithmic_bytes_per_launch": per_launch, "avg_launch_us": launch_us,
                "peak_source": ("MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
                                else "fallback 6.8 TB/s (of fallback)"),
                "note": "population of 0.8 MB stays in L2; the generation loop is latency-bound"}
    roof["avg_generation_us"] = avg_gen_us

    line = {"metric": METRIC, "value": value, "unit": "trial evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[prec_name], "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": prec_name, "generations": G, "fp64_band": "near-optimum",
                       "kernel_path": KERNEL_PATH_NAMES[path],
                       "l2": "flushed between runs (512 MiB write)", "parallelism": f"replicas x{world}"},
            "generations_per_s": world * G * args.steps / (dev_ms / 1e3), "best_f_last_run": head["best_f"],
            "forms": forms, "wall_s": t_wall, "e2e": e2e, "roofline": roof, "clocks": clk,
            "fp64_rate_tflops_measured": fp64_peak,
            "gpu_launches": args.steps * launches_per_step(head["plan"], G)}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(*make_problem())
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- other workloads
def _timed(torch, stream, flush, steps, warmup, fn):
    """Device time (ms) of `steps` calls of fn, after `warmup` calls; L2 flushed
    between calls outside the events."""
    for _ in range(warmup):
        fn()
        flush.zero_()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in evs:
        e0.record(stream)
        fn()
        e1.record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in evs)


def run_workload(args, capi, torch, rank, world):
    """The batched (512 uneven runs), surrogate (ODE, k = 8) and stress
    (NP = 8192, D = 1000) configurations; one JSON line each."""
    from paper_2405_16551_gb300 import problems

    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    steps, warmup = args.steps, args.warmup
    line = {"n_gpus": world, "steps": steps, "warmup": warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "unit": "trial evals/s"}
    if args.workload == "sphere_small":
        # the small FP64 sphere run: NP = 64, D = 10, up to 1000 generations, stop at 1e-8
        o = problems.shift(10, seed=1)
        c = capi.make_config(64, 10, objective=0, shift=o, seed=1, max_generations=1000, target_error=1e-8)
        h = capi.de_init(c, stream=stream.cuda_stream)
        gens = []

        def one():
            capi.de_reset(h)
            capi.de_run(h)

        ms = _timed(torch, stream, flush, steps, warmup, one)
        r = capi.de_get_best(h)
        capi.de_destroy(h)
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        _, _, go, evo, _ = oracle.run(64, 10, 0.5, 0.9, -100.0, 100.0, 0, o, None, seed=1, max_generations=1000,
                                      target_error=1e-8)
        cpu_s = time.perf_counter() - t0
        line.update(metric="trial evals/sec, NP=64 D=10 shifted sphere FP64, run to 1e-8 (at most 1000 generations)",
                    value=64 * r["generations"] * steps / (ms / 1e3), ms_per_step=ms / steps, dtype="f64",
                    config={"workload": "NP=64 D=10 sphere, seed 1, stop at 1e-8", "generations": r["generations"],
                            "l2": "flushed between steps (512 MiB write)"},
                    cpu_baseline={"value": 64 * go / cpu_s, "unit": "trial evals/s", "cores": 1, "kind": "oracle",
                                  "sample": f"the whole run ({go} generations, {evo} evaluations), one thread"},
                    gpu_launches=None)
    elif args.workload == "batch512":
        G = min(args.generations, 200)
        shapes = problems.batch_shapes(512, seed=1)
        forms = {}
        for name in ("bf16x3", "fp64"):
            cfgs = []
            for r, (n, d, obj) in enumerate(shapes):
                cfgs.append(capi.make_config(n, d, objective=obj, shift=problems.shift(d, seed=1, run_id=r),
                                             rot=problems.rotation(d, seed=1, run_id=r), seed=1, run_id=r,
                                             precision=PREC_NAMES[name], target_error=0.0, max_generations=G))
            h = capi.de_init_batch(cfgs, stream=stream.cuda_stream)
            path = capi.de_get_plan(h)["kernel_path"]
            ms = _timed(torch, stream, flush, steps, warmup, lambda: (capi.de_reset(h, -1), capi.de_step(h, G)))
            capi.de_destroy(h)
            tot = sum(n for n, _, _ in shapes) * G * steps
            forms[name] = {"trial_evals_per_s": tot / (ms / 1e3), "ms_per_step": ms / steps,
                           "kernel_path": KERNEL_PATH_NAMES[path]}
        # the same runs one handle at a time in plain FP64 (first 16 runs, scaled by their share of the trials)
        ms_seq, tr_seq = 0.0, 0
        for r, (n, d, obj) in enumerate(shapes[:16]):
            c = capi.make_config(n, d, objective=obj, shift=problems.shift(d, seed=1, run_id=r),
                                 rot=problems.rotation(d, seed=1, run_id=r), seed=1, run_id=r, target_error=0.0,
                                 max_generations=G)
            h = capi.de_init(c, stream=stream.cuda_stream)
            ms_seq += _timed(torch, stream, flush, 1, 1, lambda: (capi.de_reset(h), capi.de_step(h, G)))
            tr_seq += n * G
            capi.de_destroy(h)
        forms["fp64_one_run_at_a_time"] = {"trial_evals_per_s": tr_seq / (ms_seq / 1e3)}
        for k in forms:
            forms[k]["speedup_vs_fp64_one_run_at_a_time"] = (forms[k]["trial_evals_per_s"]
                                                             / forms["fp64_one_run_at_a_time"]["trial_evals_per_s"])
        line.update(metric="trial evals/sec, 512 independent runs (D in {10,30,50,100}, NP in 50..1000, 4 objectives)",
                    value=forms["bf16x3"]["trial_evals_per_s"], ms_per_step=forms["bf16x3"]["ms_per_step"],
                    dtype="bf16x3 products, f32 accumulate, f64 trials and selection band",
                    config={"workload": f"512-run batch, {G} generations per step, one handle, CUDA graphs",
                            "l2": "flushed between steps (512 MiB write)"},
                    forms=forms,
                    gpu_launches=steps * (3 * 512 + (1 if forms["bf16x3"]["kernel_path"] == KERNEL_PATH_NAMES[5]
                                                     else 3 * G)))
    elif args.workload == "ode_surrogate":
        # wall time and true evaluations to reach f < 1e-8: plain DE (k = 1)
        # against 8 screened candidates (25 Adam steps per retraining, the
        # default, and 100), 5 seeds each; then the objective cost at which
        # the surrogate would break even
        seeds = (1, 2, 3, 4, 5)
        res = {}
        for name, k, steps_tr in (("plain_k1", 0, 0), ("surrogate_k8", 8, 0), ("surrogate_k8_steps100", 8, 100)):
            runs = []
            for seed in seeds:
                c = capi.make_config(256, 20, objective=4, shift=problems.ode_hidden(seed), seed=seed,
                                     max_evals=200000, max_generations=10**6, target_error=1e-8, surrogate_k=k,
                                     surrogate_steps=steps_tr)
                h = capi.de_init(c, stream=stream.cuda_stream)
                t0 = time.perf_counter()
                r = capi.de_run(h)[0]
                runs.append({"seconds": time.perf_counter() - t0, "true_evals": r["evals"],
                             "generations": r["generations"], "best_f": r["best_f"], "stop": r["stop_reason"]})
                capi.de_destroy(h)
            res[name] = {"runs": runs, "mean_seconds": float(np.mean([r["seconds"] for r in runs])),
                         "mean_true_evals": float(np.mean([r["true_evals"] for r in runs])),
                         "mean_generations": float(np.mean([r["generations"] for r in runs]))}
        # the objective's own time per generation: NP = 256 rows through de_eval
        c = capi.make_config(256, 20, objective=4, shift=problems.ode_hidden(1), seed=1, max_generations=1)
        h = capi.de_init(c, stream=stream.cuda_stream)
        xd = torch.from_numpy(problems.population(256, 20, seed=2)).cuda()
        fd = torch.zeros(256, dtype=torch.float64, device="cuda")
        capi.de_eval(h, 0, xd.data_ptr(), 20, 256, fd.data_ptr())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            capi.de_eval(h, 0, xd.data_ptr(), 20, 256, fd.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        t_obj = e0.elapsed_time(e1) / 10 / 1e3
        capi.de_destroy(h)
        gp, wp = res["plain_k1"]["mean_generations"], res["plain_k1"]["mean_seconds"]
        for name in ("surrogate_k8", "surrogate_k8_steps100"):
            gs, ws = res[name]["mean_generations"], res[name]["mean_seconds"]
            cp, cs = wp / gp - t_obj, ws / gs - t_obj  # per-generation cost besides the objective
            res[name]["overhead_per_generation_s"] = cs - cp
            if gs < gp:
                tb = (gs * cs - gp * cp) / (gp - gs)
                res[name]["break_even_objective_s_per_generation"] = tb
                res[name]["break_even_objective_s_per_evaluation"] = tb / 256
                res[name]["break_even_vs_this_objective"] = tb / t_obj
            else:
                res[name]["break_even_objective_s_per_generation"] = None  # saves no generations
        ev = sum(r["true_evals"] for r in res["plain_k1"]["runs"])
        tm = sum(r["seconds"] for r in res["plain_k1"]["runs"])
        line.update(metric="true evaluations/sec to f < 1e-8, ODE fit (D=20, NP=256, RK4 2000 steps FP64)",
                    value=ev / tm, ms_per_step=1e3 * tm / len(seeds), dtype="f64 objective, bf16 surrogate",
                    config={"workload": "ODE fit, 5 seeds, plain DE (k = 1) and 8 screened candidates (25 or 100 "
                                        "Adam steps per retraining), budget 2e5 true evaluations"},
                    runs=res, objective_seconds_per_generation=t_obj, gpu_launches=None)
    elif args.workload == "variants":
        # the strategy variants and jDE on the FP64 path: rotated Rastrigin
        # NP = 1024, D = 100, reset + G generations per step, and the best f
        # each reaches after G generations
        G = min(args.generations, 1000)
        n, d = 1024, 100
        o, M = problems.shift(d, seed=1), problems.rotation(d, seed=1)
        forms = {}
        for name, st, jde, prec in (("rand1bin", 0, False, 0), ("best1bin", 1, False, 0), ("rand1exp", 2, False, 0),
                                    ("jde_rand1bin", 0, True, 0), ("jde_rand1exp", 2, True, 0),
                                    ("bf16x3_rand1bin", 0, False, 1), ("bf16x3_jde_rand1bin", 0, True, 1),
                                    ("bf16x3_jde_rand1exp", 2, True, 1)):
            c = capi.make_config(n, d, objective=1, shift=o, rot=M, seed=1, target_error=0.0, max_generations=G,
                                 strategy=st, jde=jde, precision=prec)
            h = capi.de_init(c, stream=stream.cuda_stream)
            ms = _timed(torch, stream, flush, steps, warmup, lambda: (capi.de_reset(h), capi.de_step(h, G)))
            b = capi.de_get_best(h)
            capi.de_destroy(h)
            forms[name] = {"trial_evals_per_s": n * G * steps / (ms / 1e3), "ms_per_step": ms / steps,
                           "us_per_generation": 1e3 * ms / steps / G, "best_f_after": b["best_f"]}
        line.update(metric="trial evals/sec, NP=1024 D=100 rotated-shifted Rastrigin, jDE (FP64), per DE variant",
                    value=forms["jde_rand1bin"]["trial_evals_per_s"], ms_per_step=forms["jde_rand1bin"]["ms_per_step"],
                    dtype="f64", config={"workload": f"NP=1024 D=100 Rastrigin, {G} generations per step, FP64 and BF16x3 forms",
                                         "l2": "flushed between steps (512 MiB write)"},
                    forms=forms, gpu_launches=None)
    elif args.workload == "suite":
        # the proposed 100-D benchmark (F01-F10) in the configuration of the
        # paper's timing study: DE/rand/1/bin, NP = 250, F = 0.5, CR = 0.3,
        # 1e7 evaluations per trial, FP64; trials batched in one handle.  Then
        # the protocol's rank-sum score of that configuration against jDE
        # (NP = 250) on the same trials' data.
        from paper_2405_16551_gb300 import protocol

        ntr = int(os.environ.get("DE_BENCH_SUITE_TRIALS", "30"))
        budget = int(float(os.environ.get("DE_BENCH_SUITE_BUDGET", "1e7")))
        d = 100
        paper_ide = [0.63, 0.61, 0.60, 0.66, 0.70, 0.78, 1.05, 1.28, 1.55, 1.85]
        algs = [protocol.Algorithm("rand1bin_np250_cr0.3", 250, f=0.5, cr=0.3),
                protocol.Algorithm("jde_np250", 250, f=0.5, cr=0.9, jde=True)]
        forms, per_fn, tot_ev, tot_s = {}, {}, 0, 0.0
        for k in range(1, 11):
            obj = problems.SUITE[k]
            data = problems.suite(obj, d, seed=1)
            # one trial alone (latency)
            t1 = protocol.run_trials(capi, algs[0], obj, d, data, 1, budget, stream=stream.cuda_stream,
                                     synchronize=torch.cuda.synchronize)[0]
            per_fn[f"F{k:02d}"] = {}
            row = {"objective": obj, "one_trial_s": t1.seconds, "one_trial_evals": t1.evals,
                   "paper_all_gpu_ide_s_rtx3080": paper_ide[k - 1]}
            for a in algs:
                tr = protocol.run_trials(capi, a, obj, d, data, ntr, budget, stream=stream.cuda_stream,
                                         synchronize=torch.cuda.synchronize)
                per_fn[f"F{k:02d}"][a.name] = tr
                secs = max(t.seconds for t in tr)
                ev = sum(t.evals for t in tr)
                row[a.name] = {"batch_s": secs, "per_trial_s": secs / ntr, "trial_evals_per_s": ev / secs,
                               "median_error": float(np.median([t.error for t in tr])),
                               "solved": sum(t.error < protocol.TARGET for t in tr)}
                if a is algs[0]:
                    tot_ev += ev
                    tot_s += secs
            forms[f"F{k:02d}"] = row
        total = protocol.benchmark_scores(per_fn)
        line.update(metric=f"trial evals/sec over the 100-D proposed benchmark F01-F10 (NP=250, CR=0.3, "
                           f"{budget:.0e} evaluations per trial, {ntr} trials batched), FP64",
                    value=tot_ev / tot_s, ms_per_step=1e3 * tot_s / 10, dtype="f64",
                    config={"workload": f"F01-F10, D=100, NP=250, F=0.5, CR=0.3, budget {budget:.0e}, {ntr} trials "
                                        "per function in one handle", "l2": "working set in L2 (a few MB)"},
                    forms=forms, protocol={"scores": total, "ranking": protocol.final_ranking(total),
                                           "algorithms": [a.name for a in algs]},
                    gpu_launches=None)
    elif args.workload == "islands":
        # the island model against one population of the same total size and
        # against the same islands without migration, on the 30-D rotated
        # Rastrigin function of the proposed benchmark (F03), at equal
        # generations and evaluations
        m, npi, d, G = 16, 64, 30, int(os.environ.get("DE_BENCH_ISLAND_GENS", "3000"))
        obj = problems.SUITE[3]
        data = problems.suite(obj, d, seed=1)
        forms = {}
        for name, kind in (("islands_ring_k20_m2", "ring"), ("islands_async_ring_k20_m2", "async"),
                           ("islands_no_migration", "none"), ("one_population_np1024", "single")):
            bests, secs = [], []
            for seed in (1, 2, 3):
                c = capi.make_config(npi if kind != "single" else m * npi, d, objective=obj, shift=data["shift"],
                                     rot=data["rot"], scale=data["scale"], seed=seed, max_generations=G,
                                     target_error=0.0)
                if kind == "single":
                    h = capi.de_init(c, stream=stream.cuda_stream)
                    nr = 1
                else:
                    h = capi.de_init_islands_ex(c, m, 1 << 30 if kind == "none" else 20, 2,
                                                capi.DE_MIGRATE_ASYNC if kind == "async" else capi.DE_MIGRATE_SYNC,
                                                stream=stream.cuda_stream)
                    nr = m
                path = KERNEL_PATH_NAMES[capi.de_get_plan(h)["kernel_path"]]
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = capi.de_run(h, nr)
                e1.record(stream)
                torch.cuda.synchronize()
                secs.append(e0.elapsed_time(e1) / 1e3)
                bests.append(min(r["best_f"] for r in res))
                capi.de_destroy(h)
            forms[name] = {"best_f_per_seed": bests, "median_best_f": float(np.median(bests)), "kernel_path": path,
                           "seconds_per_run": float(np.mean(secs)),
                           "trial_evals_per_s": m * npi * G / float(np.mean(secs))}
        line.update(metric=f"trial evals/sec, island model (16 x NP=64, ring migration every 20 generations, "
                           f"2 migrants) on the 30-D rotated Rastrigin function F03, FP64",
                    value=forms["islands_ring_k20_m2"]["trial_evals_per_s"],
                    ms_per_step=1e3 * forms["islands_ring_k20_m2"]["seconds_per_run"], dtype="f64",
                    config={"workload": f"F03 D=30, {G} generations, 3 seeds; islands (synchronous and "
                                        "asynchronous migration) vs no migration vs one population of 1024",
                            "l2": "working set in L2"},
                    forms=forms, gpu_launches=None)
    elif args.workload == "accuracy":
        line.update(accuracy_workload(capi, torch, stream, problems))
    elif args.workload == "split_error":
        line.update(split_error_workload(capi, torch, problems))
    elif args.workload == "stress_batch":
        # 64 runs of the large-dimension shape in one handle (working set far above L2)
        G = min(args.generations, 10)
        n, d, R = 8192, 1000, int(os.environ.get("DE_BENCH_BATCH_RUNS", "64"))
        cfgs = [capi.make_config(n, d, objective=1, shift=problems.shift(d, seed=1, run_id=r),
                                 rot=problems.rotation(d, seed=1, run_id=r), seed=1, run_id=r,
                                 precision=PREC_NAMES["bf16x3"], target_error=0.0, max_generations=G)
                for r in range(R)]
        h = capi.de_init_batch(cfgs, stream=stream.cuda_stream)
        ms = _timed(torch, stream, flush, steps, warmup, lambda: (capi.de_reset(h, -1), capi.de_step(h, G)))
        capi.de_destroy(h)
        value = R * n * G * steps / (ms / 1e3)
        # the trial construction's FP64 work: x_r2 - x_r3, the fused
        # multiply-add of Eq. 2 and t - o per coordinate (4 flops); its rate
        # over the whole step against the measured FP64 rate is a lower bound
        # on the trial kernel's own FP64-pipe fraction
        fp64_peak = capi.de_selftest_fp64_rate()
        trial_fp64_tflops = 4.0 * R * n * d * G * steps / (ms / 1e3) / 1e12
        line.update(metric=f"trial evals/sec, {R} runs of NP=8192 D=1000 rotated-shifted Rastrigin, BF16x3",
                    value=value, ms_per_step=ms / steps, dtype="bf16x3 products, f32 accumulate",
                    config={"workload": f"{R} x (NP=8192 D=1000), {G} generations per step, one handle",
                            "l2": f"working set about {R / 4:.0f} GB, far above L2"},
                    tensor_tflops=3 * 2.0 * R * n * d * d * G * steps / (ms / 1e3) / 1e12,
                    trial_fp64_tflops_over_step=trial_fp64_tflops, fp64_rate_tflops_measured=fp64_peak,
                    trial_fp64_frac_over_step=trial_fp64_tflops / fp64_peak,
                    hbm_frac_over_step=R * n * (2 * 8 * d + 16) * G * steps / (ms / 1e3) / 1e9 /
                    float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
                    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None,
                    gpu_launches=steps * (3 * R + 3 * G))
    else:  # stress
        G = min(args.generations, 100)
        n, d = 8192, 1000
        c = capi.make_config(n, d, objective=1, shift=problems.shift(d, seed=1), rot=problems.rotation(d, seed=1),
                             seed=1, precision=PREC_NAMES["bf16x3"], target_error=1e-8, max_generations=G)
        h = capi.de_init(c, stream=stream.cuda_stream)
        ms = _timed(torch, stream, flush, steps, warmup, lambda: (capi.de_reset(h), capi.de_step(h, G)))
        plan = capi.de_get_plan(h)
        capi.de_destroy(h)
        value = n * G * steps / (ms / 1e3)
        flops = 3 * 2.0 * n * d * d * G * steps
        line.update(metric="trial evals/sec, NP=8192 D=1000 rotated-shifted Rastrigin, BF16x3",
                    value=value, ms_per_step=ms / steps, dtype="bf16x3 products, f32 accumulate",
                    config={"workload": f"NP=8192 D=1000, {G} generations per step", "kernel_path": plan["kernel_path"],
                            "l2": "flushed between steps (512 MiB write)"},
                    tensor_tflops=flops / (ms / 1e3) / 1e12, gpu_launches=steps * (3 + 3 * G))
    line["clocks"] = clocks.stop()
    return line


def split_error_workload(capi, torch, problems):
    """Fitness error of each precision form against the FP64 oracle, per
    objective (Sec. 7.3.1: sphere, Rastrigin, Rosenbrock, Ackley) x D in
    {10, 100, 1000} x {64 random points in [-100, 100]^D, 64 points where the
    oracle's f is 1e-8 (x = o + delta v, v a random unit vector, delta by
    bisection on the oracle)}, all rotated and shifted, evaluated through
    de_eval.  Reported per cell: the largest and median |f_gpu - f| / (|f| + S)
    (the parity tolerance's scale) and the largest plain |f_gpu - f| / |f|.
    Split precision takes Rosenbrock up to D = 256 only."""
    import oracle

    oracle.build()
    n = 64
    names = {0: "sphere", 1: "rastrigin", 2: "rosenbrock", 3: "ackley"}
    forms = {"fp64": {}, "bf16x3": {}, "tf32x3": {}}
    for obj in range(4):
        for d in (10, 100, 1000):
            o, M = problems.shift(d, seed=5), problems.rotation(d, seed=5)
            rng = np.random.default_rng(1000 * obj + d)
            V = rng.normal(size=(n, d))
            V /= np.linalg.norm(V, axis=1, keepdims=True)
            lo_d, hi_d = np.zeros(n), np.ones(n)  # f(o + v) > 1e-8 for every objective here
            for _ in range(45):
                mid = 0.5 * (lo_d + hi_d)
                fm, _ = oracle.evaluate(obj, o + mid[:, None] * V, o, M)
                above = fm > 1e-8
                hi_d = np.where(above, mid, hi_d)
                lo_d = np.where(above, lo_d, mid)
            sets = {"random": problems.population(n, d, seed=11), "f_1e-8": o + hi_d[:, None] * V}
            ref = {k: oracle.evaluate(obj, X, o, M) for k, X in sets.items()}
            for form, prec in (("fp64", capi.DE_PREC_FP64), ("bf16x3", capi.DE_PREC_BF16X3),
                               ("tf32x3", capi.DE_PREC_TF32X3)):
                cell = forms[form].setdefault(names[obj], {})
                if prec != capi.DE_PREC_FP64 and obj == 2 and d > 256:
                    cell[str(d)] = "unsupported (split Rosenbrock up to D = 256)"
                    continue
                h = capi.de_init(capi.make_config(n, d, objective=obj, shift=o, rot=M, precision=prec,
                                                  max_generations=1))
                res = {}
                try:
                    for k, X in sets.items():
                        xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
                        fd = torch.zeros(n, dtype=torch.float64, device="cuda")
                        capi.de_eval(h, 0, xd.data_ptr(), d, n, fd.data_ptr())
                        torch.cuda.synchronize()
                        f = fd.cpu().numpy()
                        fo, sabs = ref[k]
                        e_tol = np.abs(f - fo) / (np.abs(fo) + sabs)
                        e_rel = np.abs(f - fo) / np.abs(fo)
                        res[k] = {"max_err_tol_scale": float(e_tol.max()), "median_err_tol_scale": float(np.median(e_tol)),
                                  "max_err_plain_relative": float(e_rel.max()), "f_median": float(np.median(fo))}
                finally:
                    capi.de_destroy(h)
                cell[str(d)] = res
    worst = {form: max(v["max_err_tol_scale"] for ob in forms[form].values() for c in ob.values()
                       if isinstance(c, dict) for v in c.values()) for form in forms}
    return dict(metric="largest fitness error of the split precisions against the FP64 oracle, |f_s - f| / (|f| + S), "
                       "objectives 0-3 x D 10/100/1000 x {random points, f = 1e-8 above the optimum}",
                value=worst["bf16x3"], unit="relative error", higher_is_better=False, ms_per_step=None,
                dtype="bf16x3 / tf32x3 products, f32 accumulate (fp64 for reference)",
                config={"workload": "64 random points and 64 points with f = 1e-8 per objective and D, "
                                    "rotated and shifted, through de_eval"},
                forms=forms, worst_err_tol_scale=worst, gpu_launches=None)


def accuracy_workload(capi, torch, stream, problems):
    """The mixed-precision and batched forms against plain FP64 GPU DE at a
    stated final error (the stopping rule of Sec. 7.3.4): wall time and true
    objective evaluations to reach it.

    * rotated sphere, NP = 1024, D = 100, F = 0.5, CR = 0.9, run to f < 1e-8
      in FP64, BF16x3 and TF32x3 (5 seeds);
    * rotated Rastrigin, the same shape: FP64 runs 3000 generations; each
      split form then runs (up to 9000 generations) until its best is below
      the FP64 run's final error (3 seeds);
    * the 512-run batch (first 32 runs, FP64, 200 generations) in one handle
      against the same runs one handle at a time: the final errors are equal
      (checked, run by run), so the comparison is the time alone.
    Times are device time (CUDA events around de_reset + de_run) and wall
    time of de_run; evaluations are NP (1 + generations), plus the split
    forms' FP64 re-evaluations, reported separately."""
    n, d = 1024, 100

    def run_to(obj, seed, prec, target, gens):
        o, M = problems.shift(d, seed=seed), problems.rotation(d, seed=seed)
        c = capi.make_config(n, d, objective=obj, shift=o, rot=M, seed=seed, precision=prec, target_error=target,
                             max_generations=gens)
        h = capi.de_init(c, stream=stream.cuda_stream)
        try:
            capi.de_run(h)  # warm-up (kernel load, autotuner cache)
            torch.cuda.synchronize()
            st0 = capi.de_get_stats(h)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            capi.de_reset(h)
            t0 = time.perf_counter()
            r = capi.de_run(h)[0]
            wall = time.perf_counter() - t0
            e1.record(stream)
            torch.cuda.synchronize()
            st = capi.de_get_stats(h)
            return {"seconds": e0.elapsed_time(e1) / 1e3, "wall_s": wall, "generations": r["generations"],
                    "evals": r["evals"], "fp64_reevals": st["fp64_reevals"] - st0["fp64_reevals"], "best_f": r["best_f"],
                    "reached": r["stop_reason"] == capi.DE_STOP_TARGET, "kernel_path": capi.de_get_plan(h)["kernel_path"]}
        finally:
            capi.de_destroy(h)

    def summary(runs):
        t = [r["seconds"] for r in runs]
        ev = [r["evals"] for r in runs]
        return {"runs": runs, "median_s": float(np.median(t)), "median_evals": float(np.median(ev)),
                "all_reached": all(r["reached"] for r in runs)}

    out = {}
    # 1. rotated sphere to 1e-8
    sph = {}
    for name in ("fp64", "bf16x3", "tf32x3"):
        sph[name] = summary([run_to(0, seed, PREC_NAMES[name], 1e-8, 20000) for seed in (1, 2, 3, 4, 5)])
    for name in sph:
        sph[name]["speedup_time_vs_fp64"] = sph["fp64"]["median_s"] / sph[name]["median_s"]
        sph[name]["evals_ratio_vs_fp64"] = sph[name]["median_evals"] / sph["fp64"]["median_evals"]
    out["rotated_sphere_to_1e-8"] = sph
    # 2. rotated Rastrigin to the FP64 run's final error after 3000 generations
    ras = {"fp64_3000_generations": [], "bf16x3": [], "tf32x3": []}
    for seed in (1, 2, 3):
        ref = run_to(1, seed, 0, 0.0, 3000)
        ras["fp64_3000_generations"].append(ref)
        for name in ("bf16x3", "tf32x3"):
            r = run_to(1, seed, PREC_NAMES[name], ref["best_f"], 9000)
            r["target"] = ref["best_f"]
            r["speedup_time_vs_fp64"] = ref["seconds"] / r["seconds"]
            r["evals_ratio_vs_fp64"] = r["evals"] / ref["evals"]
            ras[name].append(r)
    for name in ("bf16x3", "tf32x3"):
        ras[name + "_median_speedup_time"] = float(np.median([r["speedup_time_vs_fp64"] for r in ras[name]]))
        ras[name + "_median_evals_ratio"] = float(np.median([r["evals_ratio_vs_fp64"] for r in ras[name]]))
        ras[name + "_all_reached"] = all(r["reached"] for r in ras[name])
    out["rotated_rastrigin_to_fp64_final_error"] = ras
    # 3. batch vs one run at a time, equal final errors
    shapes = problems.batch_shapes(512, seed=1)[:32]
    G = 200
    cfgs = [capi.make_config(nn, dd, objective=obj, shift=problems.shift(dd, seed=1, run_id=r),
                             rot=problems.rotation(dd, seed=1, run_id=r), seed=1, run_id=r, target_error=0.0,
                             max_generations=G) for r, (nn, dd, obj) in enumerate(shapes)]
    hb = capi.de_init_batch(cfgs, stream=stream.cuda_stream)
    capi.de_run(hb, len(cfgs))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    capi.de_reset(hb, -1)
    rb = capi.de_run(hb, len(cfgs))
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    capi.de_destroy(hb)
    t_seq, same = 0.0, True
    for r, c in enumerate(cfgs):
        h = capi.de_init(c, stream=stream.cuda_stream)
        capi.de_run(h)
        torch.cuda.synchronize()
        e0.record(stream)
        capi.de_reset(h)
        rs = capi.de_run(h)[0]
        e1.record(stream)
        torch.cuda.synchronize()
        t_seq += e0.elapsed_time(e1) / 1e3
        same = same and rs["best_f"] == rb[r]["best_f"] and rs["generations"] == rb[r]["generations"]
        capi.de_destroy(h)
    out["batch_vs_one_at_a_time"] = {"runs": len(cfgs), "generations": G, "batched_s": t_batch,
                                     "one_at_a_time_s": t_seq, "speedup_time": t_seq / t_batch,
                                     "final_errors_identical": same,
                                     "trials": sum(nn for nn, _, _ in shapes) * G}
    return dict(metric="wall-time speedup over plain FP64 GPU DE to f < 1e-8, rotated sphere NP=1024 D=100 (BF16x3)",
                value=sph["bf16x3"]["speedup_time_vs_fp64"], unit="x", ms_per_step=1e3 * sph["bf16x3"]["median_s"],
                dtype="f64 / bf16x3 / tf32x3 forms compared",
                config={"workload": "rotated sphere and rotated Rastrigin NP=1024 D=100 F=0.5 CR=0.9 to a stated "
                                    "error; 32 batch runs FP64 200 generations", "l2": "working set in L2"},
                forms=out, gpu_launches=None)


# DRAM traffic of one launch of the dominant kernel, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of a 200-generation launch of
# the BF16x3 persistent kernel on this workload, scaled to a launch of 3000
# generations (traffic grows with generations); a kernel changed since its
# last capture has no entry
TRAFFIC_PER_LAUNCH = {
    # k_persist_cta, 7 targets per CTA: 986,112 + 448,000 bytes per 200 generations
    ("k_persist_cta", 3000): (986112 + 448000) * 3000 // 200}


if __name__ == "__main__":
    main()
