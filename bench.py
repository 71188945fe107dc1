#!/usr/bin/env python
"""Throughput benchmark: proton histories per second on one GB300.

Workload (default): the heterogeneous slab phantom -- 128^3 voxels of 1.5 mm
(water / cortical bone / lung / water with a 1 cm titanium insert), 1e6 protons
split over 70, 150 and 230 MeV pencil beams of sigma 4 mm, full physics with
the intranuclear cascade.  One step = one complete transport of all 1e6
histories (one graph launch: phase space and transport of the primaries, the
cascade of their non-elastic events, the drain of every later generation, then
the batch-statistics kernel), inputs resident in HBM.  The headline build is
the -use_fast_math one (the build the method's authors timed; both builds pass
the same parity tests against the oracle); the IEEE build is timed beside it.

Prints one JSON line.  `--impl reference` times the CPU oracle on a bounded
sample of the same workload instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "proton histories/s on 1 GB300, full cascade (learned surrogate reported beside it)"
UNIT = "histories/s"
N_HISTORIES = 1_000_000
# Scalar operations one condensed-history step needs (the common step: a voxel crossing
# with multiple scattering and straggling), counted from its formulas with every add,
# multiply, fused multiply-add, compare, select, conversion, integer and special-function
# instruction as one (a division as reciprocal + multiply, a square root or logarithm as
# two): Philox4x32-10 block 99, five uniforms 26, two boundary distances 78, multiple
# scattering with the direction rotation 60, straggling 20, inverse-range spline 24,
# range spline 16, fixed-point deposit 23, cross-section table and lambda 13, and the
# rest of the step logic 50.  Peak = FP32/INT32 lanes x SM clock.
OPS_PER_STEP = 409
# Algorithmic bytes of a step at L2 on the slab workload: material id 1 B + density 4 B +
# the tally's 64-bit read-modify-write 16 B.
BYTES_PER_STEP = 21
# The learned stand-in's two network passes per event (multiplicity, then the products), each
# 2 x (32*256 + 3*256*256 + 256*16) multiply-add FLOPs.
SURROGATE_FLOPS_PER_EVENT = 2 * 2 * (32 * 256 + 3 * 256 * 256 + 256 * 16)
L2_BYTES = 129 * 2 ** 20
# Measurements of the primary-transport kernel that need a profiler, valid only for the kernel
# sources they were taken on (their SHA-256 below; otherwise reported as null).
#   ncu: one ncu capture of the first primary launch of the 2e5-history slab case (-k
#        transport_kernel -c 1): issue slots busy, threads per executed instruction (SIMT
#        efficiency = that / 32) and thread instructions per condensed-history step.
#   bytes_per_history: DRAM bytes (read + write) of a full 1e6-history primary launch per
#        primary history: dram__bytes_read.sum + dram__bytes_write.sum alone (one pass), one
#        launch (-c 1): 93.59 + 7.95 MB (the reads include the 48-byte phase-space records).
KERNEL_SOURCES = ("transport.cu", "transport_step.cuh", "pmc_device.cuh", "pmc_kernels.cuh")
KERNEL_SHA256 = "5c5104197768be75e1b9d53009253bd1444afb8c5d21b1009623b929060c583e"
NCU = {"issue_slots_busy": 0.7499, "threads_per_instruction": 21.64, "thread_instructions_per_step": 553.3,
       "capture": "slab workload, 2e5 histories, first primary launch (-k regex:^transport_kernel -c 1)"}
TRAFFIC = {"bytes_per_history": 101.55}


def _sources_match():
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1409_8336_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest() == KERNEL_SHA256


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--histories", type=int, default=N_HISTORIES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--math", default="fast", choices=["fast", "ieee"], help="headline build")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--train-events", type=int, default=10_000_000)
    ap.add_argument("--no-gamma", action="store_true")
    ap.add_argument("--no-let", action="store_true")
    ap.add_argument("--no-moliere", action="store_true")
    ap.add_argument("--no-vavilov", action="store_true")
    ap.add_argument("--no-inc", action="store_true")
    ap.add_argument("--no-plans", action="store_true")
    ap.add_argument("--launch", default=None, help="BLOCK,CHUNK: fixed launch shape instead of autotuning")
    ap.add_argument("--plans-scale", type=float, default=1.0, help="histories per plan x this")
    ap.add_argument("--plans-slots", type=int, default=4)
    ap.add_argument("--plans-budget-gb", type=float, default=64.0)
    ap.add_argument("--inc-events", type=int, default=2_600_000)
    ap.add_argument("--gamma-histories", type=int, default=10_000_000)
    ap.add_argument("--no-ct", action="store_true")
    ap.add_argument("--no-other-build", action="store_true", help="skip timing the other math build")
    ap.add_argument("--ct-histories", type=int, default=10_000_000)
    ap.add_argument("--ct-steps", type=int, default=5)
    return ap.parse_args()


def traffic_per_launch(histories_per_launch):
    if TRAFFIC["bytes_per_history"] is None or not _sources_match():
        return None
    return TRAFFIC["bytes_per_history"] * histories_per_launch


def ncu_fractions():
    """The profiler's view of the primary launch beside the operation-count roofline."""
    if not _sources_match():
        return None
    return {"issue_slots_busy": NCU["issue_slots_busy"],
            "simt_efficiency": NCU["threads_per_instruction"] / 32.0,
            "thread_instructions_per_step": NCU["thread_instructions_per_step"], "capture": NCU["capture"]}


def memory_fractions(pk, steps_per_step, span_ms, traffic, launches_per_step):
    """The transport's memory side beside its ALU roofline: the algorithmic bytes of its steps
    (served mostly by L2) and the DRAM bytes ncu measured, both against the measured HBM peak."""
    hbm = float(pk.get("hbm_gbs", 6800.0))
    alg = BYTES_PER_STEP * steps_per_step / (span_ms * 1e-3) / 1e9
    out = {"peak_gbs": hbm, "algorithmic_bytes_per_step": BYTES_PER_STEP, "algorithmic_gbs": alg,
           "algorithmic_frac": alg / hbm, "dram_gbs": None, "dram_frac": None}
    if traffic is not None:
        d = traffic * launches_per_step / (span_ms * 1e-3) / 1e9
        out["dram_gbs"], out["dram_frac"] = d, d / hbm
    return out


def workload():
    from paper_1409_8336_gb300 import workloads as W

    return W.config2()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = max(mx, float(r[1]))
                for n, v in zip(names, r[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(prob, n_total, seconds, seed=1):
    """Times the CPU oracle (single thread) on an even sample of the workload's spots."""
    from oracle import oracle as O

    cnt = O.allocate_histories(prob, n_total)
    first = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    # pilot to size the sample
    t0 = time.perf_counter()
    for s in range(len(cnt)):
        O.run(prob, n_total, seed, h_begin=int(first[s]), h_end=int(first[s]) + 30)
    pilot = time.perf_counter() - t0
    per = max(1, int(seconds / max(pilot, 1e-6) * 30))
    t0 = time.perf_counter()
    done = 0
    for s in range(len(cnt)):
        k = min(per, int(cnt[s]))
        O.run(prob, n_total, seed, h_begin=int(first[s]), h_end=int(first[s]) + k)
        done += k
    dt = time.perf_counter() - t0
    return done / dt, done, dt


_ORACLE_FIELDS = None


def _oracle_init(fields):
    global _ORACLE_FIELDS
    _ORACLE_FIELDS = fields


def _oracle_range(job):
    """One worker's share: histories [h0, h1) of the workload through the oracle (totals only;
    the tally stays in the worker)."""
    from oracle import oracle as O

    n_total, seed, h0, h1 = job
    return O._run_range((_ORACLE_FIELDS, n_total, seed, h0, h1, False))[1]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The CPU oracle over all host cores: spawned worker processes (safe after CUDA has been
    initialised in this process) holding the workload, each running history ranges."""

    def __init__(self, prob, n_total, procs=None):
        import multiprocessing as mp
        from oracle import oracle as O

        self.procs = procs or host_cores()
        self.n_total = n_total
        self.cnt = O.allocate_histories(prob, n_total)
        self.first = np.concatenate([[0], np.cumsum(self.cnt)[:-1]])
        fields = {k: getattr(prob, k) for k in O._PROBLEM_FIELDS}
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init, initargs=(fields,))
        f0 = int(self.first[0])
        self.pool.map(_oracle_range, [(n_total, 1, f0, f0 + 1)] * self.procs, chunksize=1)   # load the oracle

    def rate(self, seconds, rate1, seed=1):
        """Histories/s over an even sample of the spots, sized from the single-thread rate
        rate1 to take about `seconds` on all workers."""
        per = max(self.procs, int(rate1 * seconds * self.procs / len(self.cnt)))
        jobs = []
        for s in range(len(self.cnt)):
            k = min(per, int(self.cnt[s]))
            cuts = [int(self.first[s]) + k * i // self.procs for i in range(self.procs + 1)]
            jobs += [(self.n_total, seed, cuts[i], cuts[i + 1]) for i in range(self.procs) if cuts[i + 1] > cuts[i]]
        done = sum(j[3] - j[2] for j in jobs)
        t0 = time.perf_counter()
        self.pool.map(_oracle_range, jobs, chunksize=1)
        dt = time.perf_counter() - t0
        return done / dt, done, dt

    def ranges(self, starts_counts, seed=1):
        """Histories/s of the given history ranges (first history, count), one job each."""
        jobs = [(self.n_total, seed, h0, h0 + k) for h0, k in starts_counts if k > 0]
        done = sum(j[3] - j[2] for j in jobs)
        t0 = time.perf_counter()
        self.pool.map(_oracle_range, jobs, chunksize=1)
        dt = time.perf_counter() - t0
        return done / dt, done, dt

    def close(self):
        self.pool.close()
        self.pool.join()


def config_block(prob, n):
    """The workload description shared by both arms."""
    return {"workload": prob.name, "histories_per_step": n, "spots": "70/150/230 MeV, sigma 4 mm",
            "batches": prob.n_batches, "physics": "full cascade", "l2": "flushed between steps"}


def max_over_ranks(value, dist=None):
    """The slowest rank's time (the whole job ends with it); a no-op on one process."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = workload()
    times, dones = [], []
    # the oracle on all host cores; each step is a bounded sample, sized so the whole run
    # ends within about two minutes
    rate1, _, _ = oracle_rate(prob, args.histories, 1.0)
    pool = OraclePool(prob, args.histories)
    per_step = min(max(args.cpu_seconds / 3, 0.5), 120.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        rate, done, dt = pool.rate(per_step, rate1, seed=1 + i)
        if i >= args.warmup:
            times.append(dt)
            dones.append(done)
    pool.close()
    value = sum(dones) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * args.histories / value,
            "ms_per_step_note": "extrapolated per history: each step times a bounded sample of the workload's "
                                "histories on all host cores and scales it to the step's %d" % args.histories,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block(prob, args.histories),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "sample": "%d histories per step, even over the three spots, on %d worker processes" %
                                       (sum(dones) // len(dones), pool.procs)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# Table I of the paper: seconds for 2.6e6 non-elastic interactions at 200 MeV on a GTX680
TABLE1_GTX680_S = {"O16": {"ieee": 8.39, "fast": 6.61}, "Ca40": {"ieee": 15.56, "fast": 9.77}}


def inc_leg(args, device, with_cpu):
    """The paper's INC benchmark (Table I): 2.6e6 proton-16O and proton-40Ca non-elastic
    interactions at 200 MeV through the event-generator entry point (cascade and
    evaporation on the device), device time per batch, both builds; the oracle's event
    generator on a bounded sample as the CPU baseline."""
    from paper_1409_8336_gb300 import Engine
    from paper_1409_8336_gb300 import workloads as W

    prob = W.config2()
    idx = {"O16": None, "Ca40": None}
    for i, nu in enumerate(prob.nuclides):
        name = {(8, 16): "O16", (20, 40): "Ca40"}.get((int(nu[0]), int(nu[1])))
        if name:
            idx[name] = i
    n = args.inc_events
    out = {"events": n, "energy_mev": 200.0, "paper": "Table I, GTX680 seconds", "targets": {}}
    for math in ("fast", "ieee"):
        eng = Engine(device=device, n_batches=prob.n_batches, fast_math=(math == "fast"))
        eng.load_problem(prob)
        for name, i in idx.items():
            eng.nonelastic_events(i, 200.0, n // 10, 99)
            ms = [eng.nonelastic_events(i, 200.0, n, 100 + r)["ms"] for r in range(3)]
            y = eng.nonelastic_events(i, 200.0, n, 100)
            t = statistics.median(ms) / 1e3
            row = out["targets"].setdefault(name, {})
            row[math] = {"seconds": t, "events_per_s": n / t, "paper_s": TABLE1_GTX680_S[name][math],
                         "speedup_vs_paper": TABLE1_GTX680_S[name][math] / t,
                         "protons_per_event": y["count"]["p"] / y["events"],
                         "neutrons_per_event": y["count"]["n"] / y["events"]}
        eng.close()
    if with_cpu:
        from oracle import oracle as O

        for name, (Z, A) in (("O16", (8, 16)), ("Ca40", (20, 40))):
            k = 2000
            t0 = time.perf_counter()
            O.inc_batch(Z, A, 200.0, 7, 0, k)
            dt = time.perf_counter() - t0
            out["targets"][name]["cpu_baseline"] = {
                "value": k / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
                "sample": "%d events in %.2f s" % (k, dt), "seconds_for_batch": n * dt / k}
    return out


def event_stage_ks(eng, prob, n_per_target=5000, seed=321):
    """The shipped event kernels on the same events: the learned stand-in's tensor-core event
    kernel against the cascade and evaporation kernels, per target nucleus (E uniform in
    10-250 MeV): KS statistics of the leading proton's energy / E and polar cosine, of the
    energies and cosines of the (up to four) most energetic protons, and the mean multiplicity
    (capped at four, the network's slots) of each."""
    from scipy import stats

    rng = np.random.default_rng(seed)
    out = {}
    for t, nu in enumerate(prob.nuclides):
        if nu[1] < 2:
            continue
        E = rng.uniform(10.0, 250.0, n_per_target)
        nuc = np.full(n_per_target, t, dtype=np.int32)
        res = []
        for mode in (0, 1):
            pr, _ = eng.debug_event_stage(mode, nuc, E, seed + t)
            ev = pr[:, 0].astype(np.int64)
            order = np.lexsort((-pr[:, 1], ev))
            pr, ev = pr[order], ev[order]
            first = np.r_[True, ev[1:] != ev[:-1]]
            rank = np.arange(len(ev)) - np.maximum.accumulate(np.where(first, np.arange(len(ev)), 0))
            top = pr[rank < 4]
            res.append((pr[first, 1] / E[ev[first]], pr[first, 2], top[:, 1] / E[top[:, 0].astype(np.int64)], top[:, 2],
                        float(np.minimum(np.bincount(ev, minlength=n_per_target), 4).mean())))
        (a, b) = res
        out["%d-%d" % (int(nu[0]), int(nu[1]))] = {
            "ks_leading_T": round(float(stats.ks_2samp(a[0], b[0]).statistic), 4),
            "ks_leading_cos": round(float(stats.ks_2samp(a[1], b[1]).statistic), 4),
            "ks_T": round(float(stats.ks_2samp(a[2], b[2]).statistic), 4),
            "ks_cos": round(float(stats.ks_2samp(a[3], b[3]).statistic), 4),
            "multiplicity_cascade_surrogate": [round(a[4], 3), round(b[4], 3)]}
    return out


def plans_leg(args, device, params):
    """The multi-plan stream: 64 synthetic CT plans (50-3000 spots, 70-230 MeV, phantoms
    128x128x96 to 320x320x200 at 1 mm, 1e6-1e7 histories each) through one GPU, several at
    a time within a device-memory budget; each plan's dose copied to the host when it
    completes.  Full cascade with the concurrency slots, the same with one slot (plans
    strictly one after another), and the surrogate form when a trained network is given."""
    from paper_1409_8336_gb300 import PlanStream
    from paper_1409_8336_gb300 import workloads as W

    plans = W.config5(scale=args.plans_scale)
    total = sum(n for _, n, _ in plans)
    p0 = plans[0][0]
    out = {"plans": len(plans), "histories": total, "budget_gb": args.plans_budget_gb,
           "phantoms": sorted({"%dx%dx%d" % p.shape[::-1] for p, _, _ in plans}),
           "spots_min_max": [min(len(p.spots) for p, _, _ in plans), max(len(p.spots) for p, _, _ in plans)]}
    forms = [("full_cascade", 0, args.plans_slots), ("full_cascade_one_slot", 0, 1)]
    if params is not None:
        forms.append(("surrogate", 1, args.plans_slots))
    for name, mode, slots in forms:
        s = PlanStream(device=device, slots=slots, budget_bytes=int(args.plans_budget_gb * 2 ** 30),
                       fast_math=(args.math == "fast"))
        s.load_materials(p0.nuclides, p0.materials, p0.hu_bins)
        if mode == 1:
            s.load_surrogate(params)
        s.run(plans[:2], mode, outputs=False)                 # warm-up: modules, pool
        t0 = time.perf_counter()
        rc, res = s.run(plans, mode, outputs="dose")
        wall = time.perf_counter() - t0
        s.close()
        ends = np.array([r["t_end_ms"] for r in res])
        lat = np.array([r["t_end_ms"] - r["t_admit_ms"] for r in res])
        ok = [r for r in res if r["status"] == 0]
        out[name] = {"status": rc, "slots": slots, "value": total / wall, "unit": UNIT, "seconds": wall,
                     "completion_ms_p50": float(np.percentile(ends, 50)),
                     "completion_ms_p99": float(np.percentile(ends, 99)),
                     "plan_ms_p50": float(np.percentile(lat, 50)), "plan_ms_p99": float(np.percentile(lat, 99)),
                     "plans_ok": len(ok), "max_plan_gb": max(r["device_bytes"] for r in res) / 2 ** 30}
        del res
    return out


def ct_plan_leg(args, device, stream, flush, with_cpu):
    """The batched CT plan: 256 x 256 x 160 int16 HU at 1 mm (seeded ellipsoids, 6-bin HU table),
    40 layers of 70-180 MeV x 50 spots = 2000 spots with lognormal weights, 1e7 histories in one
    graph launch with the autotuned launch shape, full cascade; L2 flushed between steps.  End to
    end through the ABI from pinned host buffers (H2D of the HU volume and spots, D2H of dose and
    error) beside it, and the oracle's per-history rate on the same plan over all host cores (a
    sample of 50 evenly spaced spots, extrapolated per history)."""
    import torch

    from paper_1409_8336_gb300 import Engine
    from paper_1409_8336_gb300 import workloads as W

    prob = W.config3()
    n = args.ct_histories
    eng = Engine(device=device, n_batches=prob.n_batches, fast_math=(args.math == "fast"))
    eng.load_problem(prob)
    block, chunk = eng.autotune(n)
    for i in range(2):
        eng.transport(n, 900 + i, stream=stream)
    ms = []
    for i in range(args.ct_steps):
        flush.fill_(float(i))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        eng.transport(n, 910 + i, stream=stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    led = eng.read_ledger()
    hu_h = torch.from_numpy(np.ascontiguousarray(prob.hu)).pin_memory()
    dose_h = torch.empty(prob.n_voxels, dtype=torch.float64).pin_memory()
    sig_h = torch.empty(prob.n_voxels, dtype=torch.float64).pin_memory()
    e2e_t = []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eng.load_phantom(prob.shape, prob.voxel, prob.origin, hu=hu_h)
        eng.clear_spots()
        eng.add_spots(prob.spots)
        eng.transport(n, 920 + i, stream=stream)
        eng.read_dose(dose_h, sig_h)
        e2e_t.append(time.perf_counter() - t0)
    eng.close()
    t = sum(ms) / len(ms)
    out = {"workload": prob.name, "histories_per_step": n, "spots": len(prob.spots), "layers": "40 x 70-180 MeV",
           "launch": {"block": block, "histories_per_subgroup": chunk or n, "autotuned": True, "graph_launches": 1},
           "value": n / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "ms_per_step_best": min(ms), "steps": len(ms),
           "e2e": {"value": n / statistics.median(e2e_t[1:]), "unit": UNIT,
                   "h2d_bytes_per_step": 2 * prob.n_voxels + 80 * len(prob.spots),
                   "d2h_bytes_per_step": 16 * prob.n_voxels},
           "steps_per_history": led["steps"] / n, "inelastic_per_history": led["inelastic"] / n}
    if with_cpu:
        pool = OraclePool(prob, n)
        # one contiguous history range per sampled spot (64 evenly spaced spots of the 2000)
        picks = list(range(0, len(prob.spots), len(prob.spots) // 64))[:64]
        target = args.cpu_seconds * 2 / 3
        rate, _, _ = pool.ranges([(int(pool.first[s]), 20) for s in picks], seed=3)      # pilot: sizes the sample
        for it in range(3):     # the pilot's per-job overhead underestimates the rate: resize until it fits
            k = max(20, int(rate * target / len(picks)))
            rate, done, dt = pool.ranges([(int(pool.first[s]), min(k, int(pool.cnt[s]))) for s in picks], seed=4 + it)
            if dt >= 0.6 * target:
                break
        pool.close()
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                               "sample": "%d histories from %d evenly spaced spots of the plan in %.1f s on %d worker "
                                         "processes, extrapolated per history" % (done, len(picks), dt, pool.procs)}
    return out


def gamma_leg(args, device, stream, flush, with_cpu):
    """The 3-D gamma index (2 %/2 mm, global, 10 % threshold) between two dose maps of the
    256 x 256 x 160 CT phantom at 1 mm from the engine at two seeds, inside the body (air
    voxels, HU < -950, set to zero as a body contour would: their dose per mass is not
    clinical): the device entry point timed with CUDA events on doses already in HBM, the
    host-array entry point end to end, and the oracle's gamma on a slab of the same maps
    as the CPU baseline."""
    import torch

    from paper_1409_8336_gb300 import Engine, GammaIndex, gamma_index
    from paper_1409_8336_gb300 import workloads as W

    prob = W.config3()
    eng = Engine(device=device, n_batches=prob.n_batches, fast_math=(args.math == "fast"))
    eng.load_problem(prob)
    maps = []
    body = prob.hu >= -950
    for seed in (11, 12):
        eng.transport(args.gamma_histories, seed, stream=stream)
        maps.append(np.where(body, eng.read_dose()[0].reshape(prob.shape), 0.0))
    eng.close()
    ref = torch.from_numpy(maps[0]).to("cuda")
    ev = torch.from_numpy(maps[1]).to("cuda")
    g = torch.empty(prob.shape, dtype=torch.float32, device="cuda")
    gi = GammaIndex(prob.voxel)
    for _ in range(3):
        gi(ref, ev, g, stream=stream)
    ms = []
    for i in range(10):
        flush.fill_(float(i))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gi(ref, ev, g, stream=stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    n_eval, n_pass = gi.counts()
    e2e = []
    for i in range(4):
        t0 = time.perf_counter()
        gamma_index(maps[0], maps[1], prob.voxel)
        e2e.append(time.perf_counter() - t0)
    nv = prob.n_voxels
    out = {"workload": "%s phantom %dx%dx%d at %g mm, %d histories per map, seeds 11 and 12" % (
               prob.name, *prob.shape[::-1], prob.voxel[0] * 10, args.gamma_histories),
           "criteria": "2 %/2 mm global, 10 % threshold, search 3 mm, on the grid", "voxels": nv,
           "evaluated": n_eval, "pass_rate": n_pass / max(n_eval, 1),
           "ms": statistics.median(ms), "voxels_per_s": nv / (statistics.median(ms) * 1e-3),
           "e2e_ms": statistics.median(e2e[1:]) * 1e3, "e2e_h2d_bytes": 16 * nv, "e2e_d2h_bytes": 4 * nv + 16,
           "kernel_bytes": 20 * nv + 8 * n_eval,
           "kernel_bytes_note": "max pass 8 B/voxel, comparison 8 B/voxel read + 4 B/voxel gamma written + "
                                "8 B per evaluated voxel of the evaluated grid"}
    out["achieved_gbs"] = out["kernel_bytes"] / (out["ms"] * 1e-3) / 1e9
    if with_cpu:
        from oracle import analysis as A

        sl = slice(prob.shape[0] // 2 - 8, prob.shape[0] // 2 + 8)
        t0 = time.perf_counter()
        A.gamma_index(maps[0][sl], maps[1][sl], prob.voxel)
        dt = time.perf_counter() - t0
        nsub = maps[0][sl].size
        out["cpu_baseline"] = {"value": nsub / dt, "unit": "voxels/s", "cores": 1, "kind": "oracle",
                               "sample": "16 central z-slices (%d voxels) of the same maps in %.2f s" % (nsub, dt)}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1409_8336_gb300 import Engine, build

    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    prob = workload()
    n = args.histories
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed_steps(eng, k, seed0):
        out = []
        for i in range(k):
            flush.fill_(float(i))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            eng.transport(n, seed0 + i, stream=stream)
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return out

    # the other build, timed beside the headline one
    fixed = args.launch is not None
    blk, chk = (int(v) for v in args.launch.split(",")) if fixed else (0, 0)
    other_ms = None
    if not args.no_other_build:
        other = Engine(device=local, n_batches=prob.n_batches, fast_math=(args.math != "fast"), block_size=blk)
        other.load_problem(prob)
        if fixed:
            other.set_launch(blk, chk)
        timed_steps(other, args.warmup, 5000)
        other_ms = timed_steps(other, args.steps, 6000)
        other.close()

    eng = Engine(device=local, n_batches=prob.n_batches, fast_math=(args.math == "fast"))
    eng.load_problem(prob)
    if fixed:
        eng.set_launch(blk, chk)
        tuned_block, tuned_chunk = blk, chk
    else:
        tuned_block, tuned_chunk = eng.autotune(n)
    # the timed steps record events around the primary-transport launches only (the
    # roofline's kernel); events around every launch cost ~3 % of a step, so the per-kind
    # breakdown comes from profiled steps after the timed region
    eng.enable_profile(True, primary_only=True)

    def one(seed):
        flush.fill_(float(seed))                           # evict L2 between steps
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        eng.transport(n, seed, stream=stream)
        b.record(stream)
        b.synchronize()
        prof, steps0 = eng.read_profile()
        return a.elapsed_time(b), prof, steps0, eng.read_ledger()

    for i in range(args.warmup):
        one(1000 + i)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, prof_ms, prof_n, steps_primary, ledgers = [], 0.0, 0, 0, []
    prof_span = 0.0
    with Clocks(local) as clk:
        for i in range(args.steps):
            t, prof, s0, led = one(rank * 100003 + i + 1)
            ms.append(t)
            prof_ms += prof["transport_primary"]["ms"]
            prof_span += prof["transport_primary"]["span_ms"]
            prof_n += prof["transport_primary"]["launches"]
            steps_primary += s0
            ledgers.append(led)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(sum(ms), dist)
    # every launch timed, on steps after the timed region (the same graph: its launch count
    # per step is the timed steps' too)
    eng.enable_profile(True)
    kinds, n_kind_steps, per_step_launches = {}, min(args.steps, 10), 0
    for i in range(n_kind_steps):
        _, prof, _, _ = one(rank * 100003 + 50000 + i)
        # the profile counts kernels (a timing pair may span two: phase space + transport,
        # cascade + evaporation, drain set-up + drain)
        per_step_launches = sum(p["kernels"] for k, p in prof.items())
        for k, v in prof.items():
            kinds.setdefault(k, [0.0, 0])
            kinds[k][0] += v["ms"] / n_kind_steps
            kinds[k][1] = v["launches"]
    eng.enable_profile(False)
    launches = per_step_launches * args.steps
    value = world * n * args.steps / (total_ms / 1e3)

    # end to end through the public API with host buffers (pinned): H2D of the phantom and spots,
    # transport, D2H of dose and error, every step
    mat_h = torch.from_numpy(np.ascontiguousarray(prob.mat)).pin_memory()
    rho_h = torch.from_numpy(np.ascontiguousarray(prob.rho)).pin_memory()
    dose_h = torch.empty(prob.n_voxels, dtype=torch.float64).pin_memory()
    sig_h = torch.empty(prob.n_voxels, dtype=torch.float64).pin_memory()
    eng.enable_profile(False)
    e2e_t = []
    for i in range(max(2, min(args.steps, 5)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eng.load_phantom(prob.shape, prob.voxel, prob.origin, mat=mat_h, rho=rho_h)
        eng.clear_spots()
        eng.add_spots(prob.spots)
        eng.transport(n, 77 + i, stream=stream)
        eng.read_dose(dose_h, sig_h)
        dt = time.perf_counter() - t0
        if i > 0:
            e2e_t.append(dt)
    e2e = world * n / statistics.median(e2e_t)
    h2d = prob.n_voxels * 5 + len(prob.spots) * 80
    d2h = prob.n_voxels * 16

    # dose-averaged LET scored beside the dose (two more tallies), timed the same way
    let_leg = None
    if not args.no_let:
        eng.enable_let(True)
        timed_steps(eng, 3, 7000)
        lm = timed_steps(eng, min(args.steps, 20), 7100)
        let_d, _ = eng.read_let()
        eng.enable_let(False)
        lval = world * n * len(lm) / (sum(lm) / 1e3)
        let_leg = {"value": lval, "unit": UNIT, "ms_per_step": sum(lm) / len(lm), "steps": len(lm),
                   "time_vs_dose_only": (sum(lm) / len(lm)) / (total_ms / args.steps),
                   "max_let_d_kev_um": float(let_d.max())}

    # Moliere multiple scattering instead of Highland, the same workload and launch shape
    moliere = None
    if not args.no_moliere:
        from paper_1409_8336_gb300 import workloads as W

        pm = prob.with_(flags=prob.flags | W.MOLIERE)
        em = Engine(device=local, n_batches=pm.n_batches, physics_flags=pm.flags, fast_math=(args.math == "fast"),
                    block_size=tuned_block)
        em.load_problem(pm)
        em.set_launch(tuned_block, tuned_chunk)
        timed_steps(em, 3, 8000)
        mm = timed_steps(em, min(args.steps, 20), 8100)
        em.close()
        moliere = {"value": world * n * len(mm) / (sum(mm) / 1e3), "unit": UNIT, "ms_per_step": sum(mm) / len(mm),
                   "steps": len(mm), "time_vs_highland": (sum(mm) / len(mm)) / (total_ms / args.steps)}

    # Vavilov straggling instead of Bohr's Gaussian, the same workload and launch shape
    vavilov = None
    if not args.no_vavilov:
        from paper_1409_8336_gb300 import workloads as W

        pv = prob.with_(flags=prob.flags | W.VAVILOV)
        ev = Engine(device=local, n_batches=pv.n_batches, physics_flags=pv.flags, fast_math=(args.math == "fast"),
                    block_size=tuned_block)
        ev.load_problem(pv)
        ev.set_launch(tuned_block, tuned_chunk)
        timed_steps(ev, 3, 8500)
        vm = timed_steps(ev, min(args.steps, 20), 8600)
        ev.close()
        vavilov = {"value": world * n * len(vm) / (sum(vm) / 1e3), "unit": UNIT, "ms_per_step": sum(vm) / len(vm),
                   "steps": len(vm), "time_vs_bohr": (sum(vm) / len(vm)) / (total_ms / args.steps)}

    # the learned stand-in of the event generator: trained outside the timed region on events
    # from the engine's own cascade, then timed the same way, with its dose against the full
    # cascade's at the same seed (2 %/2 mm gamma)
    surrogate = None
    if not args.no_surrogate:
        from paper_1409_8336_gb300 import gamma_index

        t0 = time.perf_counter()
        tr = eng.train_surrogate(n_events=args.train_events, epochs=2, batch=8192, lr=1e-3, seed=4)
        train_s = time.perf_counter() - t0
        eng.enable_profile(False)
        for i in range(args.warmup):
            eng.transport(n, 2000 + i, mode=1, stream=stream)
        sm = []
        for i in range(args.steps):
            flush.fill_(float(i))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            eng.transport(n, 3000 + i, mode=1, stream=stream)
            b.record(stream)
            b.synchronize()
            sm.append(a.elapsed_time(b))
        # the fused event stage, timed on profiled steps after the timed ones
        eng.enable_profile(True)
        ev_ms, n_ev, n_prof = 0.0, 0, min(args.steps, 10)
        for i in range(n_prof):
            flush.fill_(float(i))
            eng.transport(n, 3500 + i, mode=1, stream=stream)
            torch.cuda.synchronize()
            ev_ms += eng.read_profile()[0]["cascade"]["ms"]
            n_ev += eng.read_ledger()["surrogate_events"]
        eng.enable_profile(False)
        eng.transport(n, 77, mode=0, stream=stream)
        Df, _ = eng.read_dose()
        eng.transport(n, 77, mode=1, stream=stream)
        Ds, _ = eng.read_dose()
        _, gam = gamma_index(Df.reshape(prob.shape), Ds.reshape(prob.shape), prob.voxel, want_map=False)
        ks = event_stage_ks(eng, prob)
        sval = world * n * args.steps / (sum(sm) / 1e3)
        pk_s, src_s = peaks()
        tflops = SURROGATE_FLOPS_PER_EVENT * n_ev / (ev_ms * 1e-3) / 1e12
        tpeak = float(pk_s.get("bf16_tflops_sustained", 1700.0))
        surrogate = {"value": sval, "unit": UNIT, "ms_per_step": sum(sm) / args.steps, "speedup_vs_full": sval / value,
                     "gamma_2pct_2mm_vs_full": gam,
                     "secondary_spectra_ks": {"sample": "5000 events per target, E uniform in 10-250 MeV, the same "
                                                         "events through both event kernels", "per_target": ks},
                     "train_events": args.train_events, "train_seconds": train_s,
                     "train_loss_first_last": [tr["first_loss"], tr["last_loss"]],
                     "network": "MLP 32-256-256-256-256-16, BF16 operands on 5th-generation tensor cores (tcgen05, accumulators "
                                "in tensor memory) in the event stage and in training, FP32 accumulate",
                     "event_stage": {"bound": "tensor", "kernel": "surrogate_event_kernel", "events_per_step": n_ev / n_prof,
                                     "ms_per_step": ev_ms / n_prof, "flops_per_event": SURROGATE_FLOPS_PER_EVENT,
                                     "achieved": tflops, "peak": tpeak, "unit": "TFLOP/s", "frac": tflops / tpeak,
                                     "peak_source": "%s bf16 sustained" % src_s,
                                     "note": "two network passes per event; the stage also builds the inputs, "
                                             "conditions the outputs and emits the products.  The network generates "
                                             "the primaries' non-elastic events; the few events of later generations "
                                             "run the full cascade inside the secondary drain, as in the full-cascade "
                                             "form"}}

    inc = None
    if not args.no_inc:
        inc = inc_leg(args, local, rank == 0 and world == 1 and not args.no_cpu_baseline)

    ct = None
    if not args.no_ct:
        ct = ct_plan_leg(args, local, stream, flush, rank == 0 and world == 1 and not args.no_cpu_baseline)

    gamma = None
    if not args.no_gamma:
        gamma = gamma_leg(args, local, stream, flush, rank == 0 and world == 1 and not args.no_cpu_baseline)

    plans = None
    if not args.no_plans:
        plans = plans_leg(args, local, eng.surrogate_params() if surrogate is not None else None)

    pk, src = peaks()
    led = ledgers[-1]
    # the primary-transport launches of the two pipelined sub-groups run concurrently: the
    # throughput is their steps over the span from the first start to the last end
    steps_per_step = steps_primary / args.steps
    span_ms = prof_span / args.steps
    achieved = OPS_PER_STEP * steps_per_step / (span_ms * 1e-3) / 1e12
    steps_per_launch = steps_primary / max(prof_n, 1)
    launch_ms = prof_ms / max(prof_n, 1)
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * sm_mhz * 1e6 / 1e12       # FP32 lanes x clock, TOP/s
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate1, done1, dt1 = oracle_rate(prob, n, args.cpu_seconds)
        pool = OraclePool(prob, n)
        rate, done, dt = pool.rate(args.cpu_seconds * 2 / 3, rate1)
        pool.close()
        cpu = {"value": rate, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
               "sample": "%d histories (equal thirds of the 70/150/230 MeV spots) in %.1f s on %d worker processes"
                         % (done, dt, pool.procs),
               "single_core": {"value": rate1, "cores": 1,
                               "sample": "%d histories (equal thirds of the spots) in %.1f s" % (done1, dt1)}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "ms_per_step_best": min(ms), "ms_per_step_median": statistics.median(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config_block(prob, n),
                           launch={"block": tuned_block, "histories_per_subgroup": tuned_chunk or n,
                                   "autotuned": not fixed},
                           parallelism="replicas" if world > 1 else "single GPU"),
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "kernel": "transport_kernel (primaries)", "achieved": achieved,
                         "peak": alu_peak, "unit": "TOP/s", "frac": achieved / alu_peak,
                         "traffic": traffic_per_launch(n / max(prof_n / args.steps, 1)),
                         "peak_source": "%s sm_max_mhz x 152 SMs x 128 FP32 lanes" % src,
                         "ops_per_step": OPS_PER_STEP, "steps_per_launch": steps_per_launch,
                         "launch_ms": launch_ms, "primary_span_ms": span_ms,
                         "primary_launches_per_step": prof_n / args.steps,
                         "ncu": ncu_fractions(),
                         "memory": memory_fractions(pk, steps_per_step, span_ms,
                                                    traffic_per_launch(n / max(prof_n / args.steps, 1)),
                                                    prof_n / args.steps)},
            "clocks": clk.summary(),
            "kernels_ms_per_step": {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in kinds.items()},
            "kernels_note": "ms = summed durations of each kind's launch groups (transport_primary: phase "
                            "space + transport; cascade: cascade + evaporation of the primaries' events, or the "
                            "learned stand-in; drain: every later generation, transport and cascades, in one "
                            "launch), from %d steps after the timed region with events around every group; the "
                            "timed steps carry events around the primary-transport groups only" % n_kind_steps,
            "math": args.math,
            "surrogate": surrogate,
            "ct_plan": ct,
            "gamma": gamma,
            "inc_table1": inc,
            "plans_stream": plans,
            "let": let_leg,
            "moliere": moliere,
            "vavilov": vavilov,
            "other_build": None if other_ms is None else {
                "math": "ieee" if args.math == "fast" else "fast",
                "value": world * n * args.steps / (sum(other_ms) / 1e3), "ms_per_step": sum(other_ms) / args.steps},
            "cpu_baseline": cpu,
            "stats": {"steps_per_history": led["steps"] / n, "inelastic": led["inelastic"],
                      "elastic": led["elastic"], "secondaries": led["secondaries"],
                      "ledger_imbalance": (led["incident"] - led["deposited"] - led["escaped"] - led["binding"]) /
                      max(1, led["incident"])},
        }
        print(json.dumps(line))
    eng.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
