"""Benchmark: SHGO nuclear-attraction shell-triples/s on GB300.

Workload (one step): the full nuclear-attraction matrix V of one molecule of the high-l FP64
configuration: 32 atoms in a 20 bohr cube, Z ~ U{1..10}, one uncontracted shell per l = 0..6 on
every atom (224 shells, 1568 functions, 25,200 shell pairs), all 32 nuclei -> 806,400
shell-triples per step.  Steps cycle over seeded replicas of that distribution, all resident in
HBM before timing.  Between steps L2 is flushed by writing a 256 MiB buffer (outside the step
events).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl shgo|reference]

--impl reference times the plain CPU oracle (the Cartesian McMurchie-Davidson route) on the host
cores on the same workload, each step one replica's full V.  Under torchrun (N > 1) every rank
runs its own replicas (no collective on the data path; "replicas only") and rank 0 prints one
JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SHGO nuclear-attraction shell-triples/s per (la,lb); speedup vs plain @1e-10"
UNIT = "shell-triples/s"
WORKLOAD = "high-l FP64: 32 atoms / 20 bohr cube, one uncontracted shell per l=0..6 per atom, 32 nuclei"
# FP64 FMA rate of the GB300: 2 DFMA per cycle per SM (ncu reports a sustained peak of 304 DFMA
# thread-instructions per cycle over the 152 SMs), 2 flops each, at the SM clock.  A DFMA
# microbenchmark measured 1.20 TFLOP/s; 1.25 TFLOP/s is the nominal figure.
FP64_DFMA_PER_CLK = 304
# DRAM traffic of the coupling phase of one V of this workload (dram__bytes_read.sum +
# dram__bytes_write.sum over the 28 coupling launches of one call, from an ncu capture of the current
# kernel), or None while no capture of the current kernel exists.
COUPLING_DRAM_BYTES_PER_V = 8.25e6
COUPLING_DRAM_NOTE = ("dram__bytes_read.sum + dram__bytes_write.sum summed over the 28 k_coupling_fp64 launches of "
                      "one V (8.25 MB read, 0 B written: the coupling blocks stay in L2), "
                      "profiles/k_coupling_fp64_traffic_highl_fp64.md")


def fp64_peak_tflops(sm_mhz: float) -> float:
    return 2.0 * FP64_DFMA_PER_CLK * sm_mhz * 1e6 / 1e12


# FP32 lanes per SM (the FP32-bulk coupling kernel issues FP32 instructions of pair arithmetic).
FP32_LANES_PER_SM = 128


def fp32_lane_peak_t(sm_mhz: float) -> float:
    """FP32 lane-instructions per second (units of 1e12): 152 SMs x 128 lanes x SM clock."""
    return 152 * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12


# Iterations of the FMA microbenchmark (2048 threads per SM x 8 chains x 4 x iters FMAs): about 25 ms on
# each pipe of a GB300 at full clock.
PEAK_ITERS = {"fp64": 1536, "fp32": 98304}


def measure_fma_peak(precision: str, stream, repeats: int = 3) -> dict:
    """The FP64 or FP32 multiply-add rate of this GPU measured now (shgo_measure_fma_rate: independent
    FMA chains on every SM, CUDA events on `stream`); the best of `repeats` launches, in TFLOP/s."""
    from paper_2404_16245_gb300 import shgo
    prec = shgo.SHGO_PREC_FP64 if precision == "fp64" else shgo.SHGO_PREC_FP32_BULK
    runs = [shgo.shgo_measure_fma_rate(prec, PEAK_ITERS[precision], stream) for _ in range(repeats)]
    best = max(r[0] for r in runs)
    return {"tflops": best / 1e12, "runs_tflops": [r[0] / 1e12 for r in runs], "ms": [r[1] for r in runs]}


def f32_coupling_instructions(basis_handle, n_centers: int) -> float:
    """Useful FP32 lane-instructions of the FP32-bulk coupling kernel for one V: per live primitive pair
    and nucleus, the pair-frame offset and T (~250), one Boys form (~650), t_j (7 Lambda), the radial sums
    (16 per entry), the harmonic recursion (20 per entry) and the nucleus sums (12 per R' entry, the Dot2
    step).  The live primitive-pair count of each class is recovered from the library's FP64 flop model
    (per primitive pair and nucleus as documented with shgo_basis_class_stats)."""
    from paper_2404_16245_gb300 import shgo
    total = 0.0
    for la, lb, _trip, _integrals, f0, _f1 in shgo.shgo_basis_class_stats(basis_handle, n_centers):
        lam = la + lb
        nb = sum((lam - L) // 2 + 1 for L in range(lam + 1))
        nr = (lam + 1) * (lam + 2) * (lam + 3) // 6
        ns = (lam + 1) ** 2
        per_triple = (9 + 11 + 5 * 7 + 1 + 3 * lam + 2 * lam + 1 + 2 * (lam // 2) + 2 * (nb - lam - 1)
                      + sum(6 * l + 5 for l in range(1, lam)) + 2 * nr)
        live_pp = f0 / (per_triple * n_centers + 2 * nr) if n_centers > 0 else 0.0
        total += live_pp * n_centers * (250 + 650 + 7 * lam + 16 * nb + 20 * ns + 12 * nr)
    return total


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seeds(rank: int, replicas: int) -> list:
    """Replica indices of one rank: ranks hold disjoint, seeded replicas of the workload (the
    path shards into independent molecules, so ranks exchange nothing but the step time)."""
    return [rank * replicas + r for r in range(replicas)]


def max_over_ranks(total_ms: float, ws: int, device=None) -> float:
    """Largest timed total over the ranks (the job's wall time for the same per-rank work)."""
    if ws <= 1:
        return float(total_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "power_w_median": statistics.median(power) if power else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def oracle_rate(replicas, seconds: float, threads: int):
    """Oracle throughput on whole replicas (full V each) until `seconds` of wall time are used."""
    import oracle
    oracle.build()
    done = 0
    triples = 0
    t0 = time.perf_counter()
    while True:
        basis, C, Z = replicas[done % len(replicas)]
        oracle.nuclear_attraction(basis, C, Z, threads=threads)
        n = len(basis["l"])
        triples += n * (n + 1) // 2 * len(Z)
        done += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return triples / el, done, el


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    from paper_2404_16245_gb300 import workloads as W
    threads = os.cpu_count() or 1
    replicas = [W.config2(replica=r) for r in range(4)]
    import oracle
    oracle.build()
    for _ in range(max(0, args.warmup)):
        b, C, Z = replicas[0]
        oracle.nuclear_attraction(b, C, Z, threads=threads)
    times = []
    triples = 0
    for k in range(args.steps):
        b, C, Z = replicas[k % len(replicas)]
        t0 = time.perf_counter()
        oracle.nuclear_attraction(b, C, Z, threads=threads)
        times.append(time.perf_counter() - t0)
        n = len(b["l"])
        triples += n * (n + 1) // 2 * len(Z)
    total = sum(times)
    value = triples / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} steps, each one replica's full V (806,400 shell-triples)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def speedup_at_1e10(n_mol: int, steps: int, stream) -> dict:
    """The metric's second half on a subset of the batched workload (its first n_mol molecules, seed
    PCG64(3000)): the plain path, one molecule at a time in FP64 through shgo_nuclear_attraction, against
    the batched path (one call for all molecules, CUDA-graph replays) in FP64 and in FP32-bulk.  Each
    variant's V is compared element by element with the plain FP64 one; a variant counts toward the
    speed-up at 1e-10 when its largest absolute difference is at most 1e-10.  CUDA events on `stream`,
    `steps` timed passes after one warm pass (and the batched calls' tuning and capture calls)."""
    import torch

    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W

    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.Generator(np.random.PCG64(3000))
    mols = [W.config3_molecule(rng) for _ in range(n_mol)]
    cs = [torch.tensor(c, device=dev) for _, c, _ in mols]
    zs = [torch.tensor(z, device=dev) for _, _, z in mols]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    bases = [shgo.Basis(b) for b, _, _ in mols]
    plain = [torch.empty((B.nbf, B.nbf), dtype=torch.float64, device=dev) for B in bases]

    def run_plain():
        for i, B in enumerate(bases):
            shgo.nuclear_attraction(B, cs[i], zs[i], out=plain[i], stream=stream)

    ms_plain = timed(run_plain)
    Cb = torch.cat(cs)
    Zb = torch.cat(zs)
    res = {"subset": f"first {n_mol} molecules of the batched workload (seed PCG64(3000), "
                     f"{int(sum(len(z) for _, _, z in mols))} atoms)",
           "plain_fp64_one_at_a_time_ms": ms_plain, "variants": {}}
    vmax = max(float(v.abs().max()) for v in plain)
    for name, prec in (("batched_fp64", shgo.SHGO_PREC_FP64), ("batched_fp32bulk", shgo.SHGO_PREC_FP32_BULK)):
        batch = shgo.Batch([(b, len(z)) for b, _, z in mols], precision=prec)
        out = torch.empty(batch.out_size, dtype=torch.float64, device=dev)
        shgo.nuclear_attraction_batched(batch, Cb, Zb, out=out, stream=stream)  # tuning call
        shgo.nuclear_attraction_batched(batch, Cb, Zb, out=out, stream=stream)  # capture call
        ms = timed(lambda: shgo.nuclear_attraction_batched(batch, Cb, Zb, out=out, stream=stream))
        diff = max(float((torch.as_tensor(batch.block(out, i)) - plain[i]).abs().max()) for i in range(n_mol))
        res["variants"][name] = {"ms": ms, "speedup_vs_plain_fp64": ms_plain / ms, "max_abs_diff": diff,
                                 "within_1e-10": diff <= 1e-10}
        batch.close()
        del out
    for B in bases:
        B.close()
    ok = {k: v for k, v in res["variants"].items() if v["within_1e-10"]}
    best = max(ok, key=lambda k: ok[k]["speedup_vs_plain_fp64"]) if ok else None
    res.update({"max_abs_v": vmax, "best_within_1e-10": best,
                "speedup_at_1e-10": ok[best]["speedup_vs_plain_fp64"] if best else None,
                "screening": "not in this figure: at 1e-10 the learned mask skips little the primitive-pair "
                             "bound has not already removed (bench.py --workload screened measures it)"})
    return res


def run_shgo(args, ws, rank, local):
    import torch
    import torch.distributed as dist

    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    R = args.replicas
    reps = [W.config2(replica=k) for k in replica_seeds(rank, R)]
    prec = {"fp64": shgo.SHGO_PREC_FP64, "fp32": shgo.SHGO_PREC_FP32_BULK}[args.precision]
    bases = [shgo.Basis(b, precision=prec) for b, _, _ in reps]
    cents = [torch.tensor(C, device=dev) for _, C, _ in reps]
    chgs = [torch.tensor(Z, device=dev) for _, _, Z in reps]
    outs = [torch.empty((B.nbf, B.nbf), dtype=torch.float64, device=dev) for B in bases]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(k):
        i = k % R
        shgo.shgo_nuclear_attraction(bases[i].handle, cents[i].shape[0], cents[i].data_ptr(), chgs[i].data_ptr(),
                                     outs[i].data_ptr(), stream)

    flops, trip = shgo.shgo_basis_flops(bases[0].handle, cents[0].shape[0])
    triples_per_step = float(trip[0])
    launches_per_step = shgo.shgo_basis_launches(bases[0].handle)

    for k in range(max(3, args.warmup)):
        step(k)
    torch.cuda.synchronize()

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev_s[k].record(stream)
        step(k)
        ev_e[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(ev_s, ev_e)]
    ms_per_step = max_over_ranks(sum(step_ms), ws, dev) / args.steps
    value = ws * triples_per_step / (ms_per_step / 1e3)

    # dominant kernel: live phase timings (CUDA events on the launching stream)
    ph = np.zeros(2)
    nrep = max(3, min(R, 8))
    for i in range(nrep):
        flush.zero_()
        a, b = shgo.shgo_nuclear_attraction_timed(bases[i % R].handle, cents[i % R].shape[0],
                                                  cents[i % R].data_ptr(), chgs[i % R].data_ptr(),
                                                  outs[i % R].data_ptr(), stream)
        ph += (a, b)
    ph /= nrep
    f32 = args.precision != "fp64"
    names = ["k_coupling_f32" if f32 else "k_coupling_fp64", "k_pair_block"]
    dom = int(np.argmax(ph))
    clk = clocks.get("sm_max_mhz") or 2070.0
    # the pipe's rate measured in this run, right after the timed region (the roofline's denominator)
    pk64 = measure_fma_peak("fp64", stream)
    pk32 = measure_fma_peak("fp32", stream) if args.precision != "fp64" else None
    if f32 and dom == 0:
        # FP32-bulk coupling: FP32 lane-instructions of its pair arithmetic (one operation each)
        work = f32_coupling_instructions(bases[0].handle, cents[0].shape[0])
        achieved = work / (ph[0] / 1e3) / 1e12
        # FP32 lane-instructions per second: the measured FFMA rate counts 2 flops per FFMA instruction
        peak = pk32["tflops"] / 2.0
        roofline = {"bound": "alu", "kernel": names[0], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "peak_source": "measured in this run: shgo_measure_fma_rate FP32 (FFMA instructions per "
                                   "second, 2048 threads per SM x 8 independent chains); each FP32 instruction of "
                                   "the pair arithmetic counted as one operation (model in bench.py)",
                    "peak_derived_nominal": fp32_lane_peak_t(clk), "peak_measurements": pk32,
                    "model_fp32_instructions_per_step": work}
    else:
        achieved = flops[dom] / (ph[dom] / 1e3) / 1e12
        peak = pk64["tflops"]
        roofline = {"bound": "alu", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "traffic": COUPLING_DRAM_BYTES_PER_V if dom == 0 else None,
                    "traffic_note": COUPLING_DRAM_NOTE,
                    "peak_source": "measured in this run: shgo_measure_fma_rate FP64 (DFMA, 2048 threads per SM x "
                                   "8 independent chains, CUDA events), best of 3",
                    "peak_derived_nominal": fp64_peak_tflops(clk), "peak_measurements": pk64}
    roofline.update({"phase_ms": [float(ph[0]), float(ph[1])],
                     "phase_tflops": [float(flops[0] / ph[0] / 1e9), float(flops[1] / ph[1] / 1e9)],
                     "algorithmic_flops_per_step": [float(flops[0]), float(flops[1])]})

    # per (la, lb) class: each class's two kernels alone (classes one after another), CUDA events
    stats = shgo.shgo_basis_class_stats(bases[0].handle, cents[0].shape[0])
    cms = np.zeros((len(stats), 2))
    for i in range(nrep):
        flush.zero_()
        cms += shgo.shgo_nuclear_attraction_class_timed(bases[i % R].handle, cents[i % R].shape[0],
                                                        cents[i % R].data_ptr(), chgs[i % R].data_ptr(),
                                                        outs[i % R].data_ptr(), stream)
    cms /= nrep
    per_class = []
    for (la, lb, trip_c, ints_c, f0, f1), (m0, m1) in sorted(zip(stats, cms), key=lambda x: (-x[0][0], -x[0][1])):
        sec = (m0 + m1) / 1e3
        per_class.append({"la": la, "lb": lb, "shell_triples_per_s": trip_c / sec, "integrals_per_s": ints_c / sec,
                          "ms": m0 + m1, "tflops": (f0 + f1) / sec / 1e12,
                          "frac": (f0 + f1) / sec / 1e12 / peak})

    # the same per class on 64 replicas in one batch: one launch per kernel and class for all of them
    per_class_64 = []
    if rank == 0 and not args.no_per_class_batch:
        rb = [W.config2(replica=100 + k) for k in range(64)]
        batch = shgo.Batch([(b, len(Z)) for b, _, Z in rb])
        Cb = torch.tensor(np.concatenate([C for _, C, _ in rb]), device=dev)
        Zb = torch.tensor(np.concatenate([Z for _, _, Z in rb]), device=dev)
        outb = torch.empty(batch.out_size, dtype=torch.float64, device=dev)
        stats_b = shgo.shgo_basis_class_stats(batch.handle, 0)
        msb = np.zeros((len(stats_b), 2))
        for it in range(4):
            m = shgo.shgo_nuclear_attraction_class_timed(batch.handle, Cb.shape[0], Cb.data_ptr(), Zb.data_ptr(),
                                                         outb.data_ptr(), stream)
            if it:
                msb += m / 3
        for (la, lb, trip_c, ints_c, f0, f1), (m0, m1) in sorted(zip(stats_b, msb), key=lambda x: (-x[0][0], -x[0][1])):
            sec = (m0 + m1) / 1e3
            per_class_64.append({"la": la, "lb": lb, "shell_triples_per_s": trip_c / sec,
                                 "integrals_per_s": ints_c / sec, "ms": m0 + m1, "tflops": (f0 + f1) / sec / 1e12,
                                 "frac": (f0 + f1) / sec / 1e12 / peak})
        batch.close()
        del outb

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pin_C = [torch.tensor(C).pin_memory() for _, C, _ in reps]
        pin_Z = [torch.tensor(Z).pin_memory() for _, _, Z in reps]
        pin_V = [torch.empty((B.nbf, B.nbf), dtype=torch.float64).pin_memory() for B in bases]
        dC = [torch.empty_like(c, device=dev) for c in pin_C]
        dZ = [torch.empty_like(z, device=dev) for z in pin_Z]
        ksteps = max(3, min(args.steps, 10))
        h2d = d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(ksteps):
            i = k % R
            b = reps[i][0]
            Bh = shgo.Basis(b, precision=prec)  # host arrays -> library-owned device buffers
            dC[i].copy_(pin_C[i], non_blocking=True)
            dZ[i].copy_(pin_Z[i], non_blocking=True)
            shgo.shgo_nuclear_attraction(Bh.handle, dC[i].shape[0], dC[i].data_ptr(), dZ[i].data_ptr(),
                                         outs[i].data_ptr(), stream)
            pin_V[i].copy_(outs[i], non_blocking=True)
            torch.cuda.synchronize()
            Bh.close()
            h2d += sum(b[key].nbytes for key in ("l", "nprim", "exps", "coefs", "xyz")) + pin_C[i].nbytes + pin_Z[i].nbytes
            d2h += pin_V[i].nbytes
        el = time.perf_counter() - t0
        e2e = {"value": ws * triples_per_step * ksteps / el, "unit": UNIT, "h2d_bytes_per_step": h2d // ksteps,
               "d2h_bytes_per_step": d2h // ksteps, "steps": ksteps,
               "note": "basis upload + pinned H2D of nuclei + kernels + D2H of V, wall clock"}

    speedup = None
    if rank == 0 and ws == 1 and args.speedup_molecules > 0:
        speedup = speedup_at_1e10(args.speedup_molecules, 2, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, done, el = oracle_rate(reps, args.cpu_seconds, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{done} full replicas of the benchmark workload in {el:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "shell_triples_per_step": triples_per_step, "replicas": R,
                       "precision": args.precision,
                       "parallelism": f"replicas x{ws}", "l2": "flushed between steps (256 MiB write, outside step events)",
                       "wall_s_timed_region": wall},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "speedup_vs_plain_at_1e-10": speedup,
            "per_class": {"note": "each class's coupling + pair kernels timed alone (classes one after another); "
                                  "frac = algorithmic FP64 flops / time / peak", "classes": per_class,
                          "classes_64_replicas_batched": per_class_64},
            "gpu_launches": launches_per_step * args.steps,
        }
        print(json.dumps(line), flush=True)
    for B in bases:
        B.close()
    return 0


def run_batched(args) -> int:
    """Batched workload: the first `--molecules` molecules of the batched configuration (atom counts
    lognormal with median 30 clipped to 8..200 at 0.05 atoms/bohr^3, 40% H with 3s2p1d, heavy atoms
    5s4p3d2f1g, 1..8 primitives, exponents log-uniform [0.05, 5000]), every molecule with its own
    nuclei.  One step = all their V blocks by one batched call (a CUDA-graph replay after the tuning
    and capture calls).  The plain path computes the same molecules one at a time."""
    import torch

    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    rng = np.random.Generator(np.random.PCG64(3000))
    mols = [W.config3_molecule(rng) for _ in range(args.molecules)]
    prec = {"fp64": shgo.SHGO_PREC_FP64, "fp32": shgo.SHGO_PREC_FP32_BULK}[args.precision]
    batch = shgo.Batch([(b, len(Z)) for b, _, Z in mols], precision=prec)
    C = torch.tensor(np.concatenate([c for _, c, _ in mols]), device=dev)
    Z = torch.tensor(np.concatenate([z for _, _, z in mols]), device=dev)
    out = torch.empty(batch.out_size, dtype=torch.float64, device=dev)
    flops, trip = shgo.shgo_basis_flops(batch.handle, 0)
    triples = float(trip[0])
    t0 = time.perf_counter()
    shgo.nuclear_attraction_batched(batch, C, Z, out=out, stream=stream)  # tuning call
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    for _ in range(max(3, args.warmup)):
        shgo.nuclear_attraction_batched(batch, C, Z, out=out, stream=stream)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(args.steps):
        shgo.nuclear_attraction_batched(batch, C, Z, out=out, stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    # plain path: one molecule at a time through the single-molecule entry point.  Bases are made, timed and
    # freed 32 molecules at a time (basis creation outside the events), so that large subsets fit the device;
    # the plain time is the sum of the groups' event times.
    cs = [torch.tensor(c, device=dev) for _, c, _ in mols]
    zs = [torch.tensor(z, device=dev) for _, _, z in mols]

    def plain_pass(precision, group=32):
        total, diff, vmax = 0.0, 0.0, 0.0
        for g0 in range(0, len(mols), group):
            idx = list(range(g0, min(len(mols), g0 + group)))
            bases = [shgo.Basis(mols[i][0], precision=precision) for i in idx]
            outs = [torch.empty((B.nbf, B.nbf), dtype=torch.float64, device=dev) for B in bases]
            for k, i in enumerate(idx):
                shgo.nuclear_attraction(bases[k], cs[i], zs[i], out=outs[k], stream=stream)
            torch.cuda.synchronize()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            for k, i in enumerate(idx):
                shgo.nuclear_attraction(bases[k], cs[i], zs[i], out=outs[k], stream=stream)
            e[1].record(stream)
            torch.cuda.synchronize()
            total += e[0].elapsed_time(e[1])
            for k, i in enumerate(idx):
                diff = max(diff, float((torch.as_tensor(batch.block(out, i)) - outs[k]).abs().max()))
                vmax = max(vmax, float(outs[k].abs().max()))
            for B in bases:
                B.close()
        return total, diff, vmax

    ms_plain, maxdiff, _ = plain_pass(prec)
    vs64 = None
    if args.precision != "fp64":
        # the plain method in FP64, one molecule at a time: the reference of the speed-up at 1e-10
        ms64, d64, vmax = plain_pass(shgo.SHGO_PREC_FP64)
        vs64 = {"ms": ms64, "value": triples / (ms64 / 1e3), "speedup_batched_vs_plain_fp64": ms64 / ms,
                "max_abs_diff_vs_fp64": d64, "max_abs_v": vmax}
    line = {"metric": METRIC, "value": triples / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": f"batched: {len(mols)} molecules of the batched configuration",
                       "shell_triples_per_step": triples, "primitive_triples_per_step": float(trip[1]),
                       "atoms": int(sum(len(z) for _, _, z in mols)), "precision": args.precision,
                       "tuning_call_s": tune_s},
            "plain_one_at_a_time": {"ms": ms_plain, "value": triples / (ms_plain / 1e3),
                                    "speedup_batched_vs_plain": ms_plain / ms, "max_abs_diff": maxdiff},
            "plain_fp64_one_at_a_time": vs64,
            "phase_flops": [float(flops[0]), float(flops[1])],
            "achieved_tflops": float(flops.sum()) / (ms / 1e3) / 1e12}
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


def run_esp(args) -> int:
    """Electrostatic potential of a density on a grid of points around the benchmark molecule (32 atoms,
    l <= 6): a seeded symmetric density, points uniform in the molecule's box padded by 4 bohr.
    One step = phi at all points (the adjoint pass over the density and the per-point pass); then the
    gradient at the same points.  L2 flushed (256 MiB write, outside the step events) before every step."""
    import torch

    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    b, C, Z = W.config2()
    B = shgo.Basis(b)
    rng = np.random.default_rng(7000)
    d = rng.normal(size=(B.nbf, B.nbf))
    D = torch.tensor((d + d.T) / 2, device=dev)
    X = torch.tensor(rng.uniform(-4.0, 24.0, (args.points, 3)), device=dev)
    phi = torch.empty(args.points, dtype=torch.float64, device=dev)
    grad = torch.empty((args.points, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev)
    steps = max(1, min(args.steps, 50))

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs]))

    peak = measure_fma_peak("fp64", stream)["tflops"]
    sampler = ClockSampler(0)
    sampler.start()
    ms = timed(lambda: shgo.esp(B, D, X, out=phi, stream=stream))
    ms_g = timed(lambda: shgo.esp_gradient(B, D, X, out=grad, stream=stream))
    clocks = sampler.stop()
    fp = shgo.shgo_basis_esp_flops(B.handle, args.points, False)
    fg = shgo.shgo_basis_esp_flops(B.handle, args.points, True)
    ach = float(fp.sum()) / (ms / 1e3) / 1e12
    ach_g = float(fg.sum()) / (ms_g / 1e3) / 1e12
    npairs = B.npairs
    line = {"metric": "electrostatic potential points/s", "value": args.points / (ms / 1e3), "unit": "points/s",
            "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"potential of a density of the 32-atom l <= 6 basis at {args.points} points",
                       "shell_pairs": npairs, "shell_pair_points_per_s": npairs * args.points / (ms / 1e3),
                       "l2": "flushed between steps (256 MiB write, outside step events)"},
            "roofline": {"bound": "alu", "kernel": "whole potential call (k_esp_fp64 per class after k_esp_adjoint)",
                         "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                         "model_tflop": [float(fp[0]) / 1e12, float(fp[1]) / 1e12],
                         "peak_source": "shgo_measure_fma_rate in this run (of measured)"},
            "gradient": {"ms_per_step": ms_g, "points_per_s": args.points / (ms_g / 1e3), "achieved_tflops": ach_g,
                         "frac": ach_g / peak, "model_tflop": [float(fg[0]) / 1e12, float(fg[1]) / 1e12]},
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    B.close()
    return 0


def run_overlap(args) -> int:
    """Overlap matrix S of the benchmark molecule's basis (32 atoms, one uncontracted shell per l = 0..6 per
    atom, 1568 functions): one step = the whole matrix, both triangles.  The arithmetic per shell pair is a few
    hundred operations, so the kernel is rated against HBM for the matrix it writes."""
    import torch

    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W
    b, _, _ = W.config2()
    B = shgo.Basis(b)
    stream = torch.cuda.current_stream()
    out = torch.empty((B.nbf, B.nbf), dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda")  # 256 MiB, larger than L2
    for _ in range(max(3, args.warmup)):
        shgo.overlap(B, out=out, stream=stream)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 200))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        shgo.overlap(B, out=out, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs]))
    written = float(B.nbf) * B.nbf * 8
    peaks = {}
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = written / (ms / 1e3) / 1e9
    line = {"metric": "overlap shell pairs/s", "value": B.npairs / (ms / 1e3), "unit": "shell-pairs/s",
            "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"overlap of the high-l benchmark basis: {len(b['l'])} shells, {B.nbf} functions",
                       "shell_pairs": B.npairs, "l2": "flushed between steps (256 MiB write, outside step events)"},
            "roofline": {"bound": "hbm", "kernel": "k_overlap", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "note": "bytes of the matrix written (both triangles) per step; the inputs are a few KB",
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"}}
    print(json.dumps(line), flush=True)
    B.close()
    return 0


def run_deriv(args) -> int:
    """Derivative integrals of the benchmark molecule (32 atoms, one uncontracted shell per l = 0..6 per atom):
    one step = dV/d(basis-function centres) for all nbf^2 elements and three components (the ket's derivative
    is the transposed element), then separately the field integrals sum_C Z_C dV/dC.  V itself is timed in
    the same run for the ratio.  L2 flushed (256 MiB write outside the events) before every step."""
    import torch

    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    b, C, Z = W.config2()
    B = shgo.Basis(b)
    Cd, Zd = torch.tensor(C, device=dev), torch.tensor(Z, device=dev)
    V = torch.empty((B.nbf, B.nbf), dtype=torch.float64, device=dev)
    D = torch.empty((3, B.nbf, B.nbf), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev)
    steps = max(1, min(args.steps, 200))

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs]))

    peak = measure_fma_peak("fp64", stream)["tflops"]
    sampler = ClockSampler(0)
    sampler.start()
    ms_v = timed(lambda: shgo.nuclear_attraction(B, Cd, Zd, out=V, stream=stream))
    ms_d = timed(lambda: shgo.nuclear_attraction_deriv(B, Cd, Zd, out=D, stream=stream))
    ms_f = timed(lambda: shgo.nuclear_field(B, Cd, Zd, out=D, stream=stream))
    rng = np.random.default_rng(7100)
    p = rng.normal(size=(B.nbf, B.nbf))
    P = torch.tensor((p + p.T) / 2, device=dev)
    G = torch.empty((B.n_shells, 3), dtype=torch.float64, device=dev)
    ms_g = timed(lambda: shgo.nuclear_attraction_gradient(B, P, Cd, Zd, out=G, stream=stream))
    clocks = sampler.stop()
    fd = shgo.shgo_basis_deriv_flops(B.handle, len(Z), False)
    ff = shgo.shgo_basis_deriv_flops(B.handle, len(Z), True)
    triples = float(B.npairs) * len(Z)
    ach_d = float(fd.sum()) / (ms_d / 1e3) / 1e12
    ach_f = float(ff.sum()) / (ms_f / 1e3) / 1e12
    line = {"metric": "derivative shell-triples/s", "value": triples / (ms_d / 1e3), "unit": "shell-triples/s",
            "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms_d, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"dV/dA, dV/dB of the high-l benchmark basis: {len(b['l'])} shells, {B.nbf} "
                                   f"functions, {len(Z)} nuclei", "shell_pairs": B.npairs,
                       "l2": "flushed between steps (256 MiB write, outside step events)"},
            "v_ms": ms_v, "deriv_over_v": ms_d / ms_v,
            "gradient": {"ms_per_step": ms_g, "over_v": ms_g / ms_v,
                         "what": "sum_ab (P_ab + P_ba) dV_ab/dA per shell for a seeded symmetric density, no matrix written"},
            "field": {"ms_per_step": ms_f, "shell_triples_per_s": triples / (ms_f / 1e3), "over_v": ms_f / ms_v,
                      "model_tflop": float(ff.sum()) / 1e12, "achieved_tflops": ach_f, "frac": ach_f / peak},
            "roofline": {"bound": "alu", "kernel": "whole derivative call (coupling at la + lb + 1, variant passes, "
                                                    "combine)", "achieved": ach_d, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach_d / peak, "traffic": None, "model_tflop": [float(fd[0]) / 1e12, float(fd[1]) / 1e12],
                         "peak_source": "shgo_measure_fma_rate in this run (of measured)"},
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    B.close()
    return 0


def run_shard(args, ws: int, rank: int, local: int) -> int:
    """One benchmark molecule's V split over the ranks (shgo_basis_create_shard: each rank takes its share of
    every class's shell pairs by primitive-pair count and writes its disjoint blocks; no collective, the host
    would gather).  value = the whole V's shell triples / the slowest rank's time per V: strong scaling.
    L2 flushed between steps."""
    import torch

    import torch.distributed as dist

    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    b, C, Z = W.config2()
    B = shgo.Basis(b, shard=(rank, ws))
    Cd, Zd = torch.tensor(C, device=dev), torch.tensor(Z, device=dev)
    out = torch.zeros((B.nbf, B.nbf), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev)
    triples = float(len(b["l"]) * (len(b["l"]) + 1) // 2) * len(Z)
    for _ in range(max(3, args.warmup)):
        shgo.nuclear_attraction(B, Cd, Zd, out=out, stream=stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        shgo.nuclear_attraction(B, Cd, Zd, out=out, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = max_over_ranks(sum(a.elapsed_time(b_) for a, b_ in evs), ws, dev) / args.steps
    if rank == 0:
        print(json.dumps({"metric": "SHGO nuclear-attraction shell-triples/s, one V split over ranks",
                          "value": triples / (ms / 1e3), "unit": "shell-triples/s", "n_gpus": ws, "steps": args.steps,
                          "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "high-l FP64 benchmark molecule, shell pairs split over the ranks",
                                     "shell_pairs_this_rank": B.npairs, "parallelism": f"pair shards x{ws}",
                                     "l2": "flushed between steps (256 MiB write, outside step events)"}}),
              flush=True)
    B.close()
    return 0


def _cluster(seed: int, n_atoms: int):
    """Screening workload: atoms uniform at 0.1 atoms/bohr^3, Z ~ U{1..9}, 4s3p2d1f on every atom
    with 1..6 primitives, exponents log-uniform [0.05, 5000]."""
    from paper_2404_16245_gb300 import workloads as W
    rng = np.random.Generator(np.random.PCG64(seed))
    box = (n_atoms / 0.1) ** (1 / 3)
    return W.molecule(rng, n_atoms, box, 1, 9, lambda Z: [0] * 4 + [1] * 3 + [2] * 2 + [3],
                      lambda r: r.integers(1, 7), 0.05, 5000.0)


def run_screened(args) -> int:
    """Learned screening on one cluster of the screening recipe, three variants side by side, all with
    the block-sparse output (only shell pairs with a primitive pair above the elementwise bound store a
    block): (a) no screening at all (SHGO_FLAG_NO_PRIM_BOUND: every primitive pair whose K_AB does not
    underflow), (b) the primitive-pair bound alone (the default plain method), (c) the bound plus the
    learned per-(shell pair, nucleus) mask, whose build is timed and charged to it.  The network is trained
    on the plain method's blocks of another cluster of the same size; its margin is calibrated on held-out
    triples; each variant's V is compared with (a) over the blocks (b) stores, and 1% of the skipped triples
    are audited with the plain method."""
    import torch

    from paper_2404_16245_gb300 import screening as S
    from paper_2404_16245_gb300 import shgo

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    # training set from the plain method on a different cluster
    t0 = time.perf_counter()
    tb, tC, tZ = _cluster(4001, args.train_atoms)
    Bt = shgo.Basis(tb)
    a, b = shgo.pair_shells(Bt.handle, Bt.npairs)
    rng = np.random.default_rng(4001)
    dist = np.linalg.norm(tb["xyz"][a] - tb["xyz"][b], axis=1)
    tr = S.sample_triples(rng, Bt.npairs, len(tZ), args.train_triples, pair_dist=dist)
    T = S.plain_labels(tb, a, b, tC, tZ, tr)
    X = shgo.screen_features(Bt.handle, torch.tensor(tC, device=dev), torch.tensor(tZ, device=dev),
                             torch.tensor(tr, device=dev))
    label_s = time.perf_counter() - t0
    nval = max(1, len(tr) // 10)
    Tt = torch.tensor(T, dtype=torch.float32, device=dev)
    t1 = time.perf_counter()
    net, losses = S.train(X[nval:].contiguous(), Tt[nval:].contiguous(), epochs=args.epochs, batch=4096, log=log)
    train_s = time.perf_counter() - t1
    Bt.close()
    Xv = X[:nval].contiguous().clone()
    del X, Tt
    # evaluation cluster
    basis, C, Z = _cluster(4000, args.atoms)
    threshold = args.threshold if args.threshold > 0 else args.target_error / len(Z)
    margin = S.calibrate_margin(net, Xv, T[:nval], math.log10(threshold), safety=2.0) \
        if args.margin <= 0 else math.log10(args.margin)
    del Xv
    Cd, Zd = torch.tensor(C, device=dev), torch.tensor(Z, device=dev)
    prec = shgo.SHGO_PREC_FP64 if args.precision == "fp64" else shgo.SHGO_PREC_FP32_BULK
    Bn = shgo.Basis(basis, precision=prec, flags=shgo.SHGO_FLAG_BLOCK_SPARSE | shgo.SHGO_FLAG_NO_PRIM_BOUND)
    Bb = shgo.Basis(basis, precision=prec, flags=shgo.SHGO_FLAG_BLOCK_SPARSE)

    def timed(fn, steps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    out_n = torch.empty(Bn.out_shape(), dtype=torch.float64, device=dev)
    out_b = torch.empty(Bb.out_shape(), dtype=torch.float64, device=dev)
    out_s = torch.empty(Bb.out_shape(), dtype=torch.float64, device=dev)
    ms_n = timed(lambda: shgo.nuclear_attraction(Bn, Cd, Zd, out=out_n, stream=stream), args.steps)
    ms_b = timed(lambda: shgo.nuclear_attraction(Bb, Cd, Zd, out=out_b, stream=stream), args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    kept, skipped = shgo.screen_build(Bb.handle, net, Cd, Zd, len(Z), math.log10(threshold), margin)
    e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    ms_s = timed(lambda: shgo.nuclear_attraction_screened(Bb.handle, Cd, Zd, len(Z), out_s, stream=stream),
                 args.steps)
    # errors against (a) over the blocks (b) stores
    _, _, off_n = shgo.shgo_sparse_layout(Bn.handle)
    _, _, off_b = shgo.shgo_sparse_layout(Bb.handle)
    pa, pb = shgo.pair_shells(Bb.handle, Bb.npairs)
    lv = np.asarray(basis["l"])
    sizes = (2 * lv[pa] + 1) * (2 * lv[pb] + 1)
    idx_b = np.concatenate([np.arange(o, o + n) for o, n in zip(off_b[off_b >= 0], sizes[off_b >= 0])])
    idx_n = np.concatenate([np.arange(o, o + n) for o, n in zip(off_n[off_b >= 0], sizes[off_b >= 0])])
    vn = out_n.cpu().numpy()
    ref = vn[idx_n]
    err_b = float(np.max(np.abs(out_b.cpu().numpy()[idx_b] - ref)))
    err_s = float(np.max(np.abs(out_s.cpu().numpy()[idx_b] - ref)))
    only_n = (off_n >= 0) & (off_b < 0)
    omitted = float(max((np.max(np.abs(vn[o:o + n])) for o, n in zip(off_n[only_n], sizes[only_n])), default=0.0))
    mask = shgo.screen_mask(Bb.handle, kept + skipped)
    rep = S.audit(basis, pa, pb, C, Z, mask, np.full(Bb.npairs, len(Z)), args.audit, np.random.default_rng(7),
                  threshold)
    fl_n, trip = shgo.shgo_basis_flops(Bn.handle, len(Z))
    fl_b, _ = shgo.shgo_basis_flops(Bb.handle, len(Z))
    value = float(trip[0]) / ((build_ms + ms_s) / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "ms_per_step": build_ms + ms_s, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == shgo.SHGO_PREC_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": f"learned screening: {args.atoms}-atom cluster at 0.1 atoms/bohr^3, 4s3p2d1f, "
                                   f"1-6 primitives, exponents log-uniform [0.05, 5000], Z ~ U{{1..9}}",
                       "precision": args.precision, "shell_triples": float(trip[0]),
                       "shell_pairs": Bb.npairs, "nbf": Bb.nbf,
                       "target_max_error": args.target_error, "per_triple_threshold": threshold,
                       "margin_log10": margin,
                       "output": "block-sparse (shgo_sparse_layout)"},
            "variants": {
                "no_screening": {"ms": ms_n, "shell_triples_per_s": float(trip[0]) / (ms_n / 1e3),
                                 "blocks_stored": int((off_n >= 0).sum()), "coupling_flops": float(fl_n[0]),
                                 "largest_element_of_blocks_the_bound_omits": omitted},
                "primitive_pair_bound": {"ms": ms_b, "shell_triples_per_s": float(trip[0]) / (ms_b / 1e3),
                                         "speedup_vs_no_screening": ms_n / ms_b,
                                         "blocks_stored": int((off_b >= 0).sum()), "coupling_flops": float(fl_b[0]),
                                         "max_abs_error_vs_no_screening": err_b},
                "bound_plus_learned_mask": {"ms_including_build": build_ms + ms_s, "build_ms": build_ms,
                                            "screened_ms": ms_s, "kept_triples": kept, "skipped_triples": skipped,
                                            "skipped_fraction": skipped / max(1, kept + skipped),
                                            "speedup_vs_no_screening": ms_n / (build_ms + ms_s),
                                            "speedup_vs_bound_alone": ms_b / (build_ms + ms_s),
                                            "speedup_vs_bound_alone_reusing_mask": ms_b / ms_s,
                                            "max_abs_error_vs_no_screening": err_s, "audit": rep}},
            "memory": {"dense_V_bytes": 8 * Bb.nbf ** 2, "block_sparse_V_bytes": 8 * Bb.ndoubles,
                       "blocks_stored": Bb.nblocks},
            "training": {"triples": int(len(tr)), "train_atoms": args.train_atoms, "epochs": args.epochs,
                         "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1], "label_s": label_s,
                         "train_s": train_s}}
    print(json.dumps(line), flush=True)
    Bn.close()
    Bb.close()
    net.close()
    return 0


def _sweep_oracle_blocks(job):
    """Oracle blocks <a|Z/|r - C||b> of precision-sweep triples (runs in a spawned worker process):
    job = (rows [k, 11] of la, lb, alpha, beta, B, C, Z; "f64" or "ld")."""
    import oracle
    from paper_2404_16245_gb300 import workloads as W
    rows, precision = job
    out = []
    for r in rows:
        la, lb = int(r[0]), int(r[1])
        basis = W.make_basis([la, lb], [1, 1], [r[2], r[3]], [1.0, 1.0], [np.zeros(3), r[4:7]])
        V = oracle.nuclear_attraction(basis, r[7:10].reshape(1, 3), r[10:11], precision=precision)
        out.append(V[:2 * la + 1, 2 * la + 1:].copy())
    return out


def run_precision_sweep(n_triples: int, n_oracle: int, n_ext: int = 100, chunk: int = 250_000) -> int:
    """Precision sweep over n_triples independent primitive triples (la, lb <= 8, exponents log-uniform
    [0.01, 1000], |AB|, |PC| <= 15, Z <= 20).  Every triple runs through the batched entry point in FP64,
    FP32-bulk and FP32-plain (one molecule per triple, `chunk` molecules per batch); per (la, lb) class the
    block-normwise error max|x - y| / max|y| of the FP32 forms against FP64, and of FP64 against the oracle
    in double on the first n_oracle triples of each class and in extended precision (binary128 on the
    aarch64 host, 80-bit on x86-64) on the first n_ext.  The oracle runs in a pool of spawned processes, one
    per host core, started before any GPU work.  Prints one JSON line."""
    import multiprocessing as mp

    import oracle
    from paper_2404_16245_gb300 import workloads as W

    t_start = time.perf_counter()
    la, lb, alpha, beta, B, C, Z = W.config5_arrays(n_triples)
    rows = np.column_stack([la, lb, alpha, beta, B, C, Z]).astype(np.float64)
    cls = la * 9 + lb
    sub_f64, sub_ext = {}, {}
    for k in range(81):
        idx = np.nonzero(cls == k)[0]
        sub_f64[k] = idx[:n_oracle]
        sub_ext[k] = idx[:n_ext]
    oracle.build()
    ncpu = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(ncpu)

    def submit(sub, precision):
        order = np.concatenate([sub[k] for k in range(81)])
        parts = np.array_split(order, max(1, 8 * ncpu))
        return order, pool.map_async(_sweep_oracle_blocks, [(rows[p], precision) for p in parts])

    ord_f64, job_f64 = submit(sub_f64, "f64")
    ord_ext, job_ext = submit(sub_ext, "ld")

    import torch

    from paper_2404_16245_gb300 import shgo
    dev = torch.device("cuda", 0)
    keep = set(np.concatenate([ord_f64, ord_ext]).tolist())
    fp64_blocks = {}
    errs = {k: {"bulk": [], "plain": []} for k in range(81)}

    def rel(g, r, floor):
        s = np.max(np.abs(r), axis=(1, 2))
        d = np.max(np.abs(g - r), axis=(1, 2))
        ok = s > floor
        return d[ok] / s[ok]

    t_gpu = 0.0
    for c0 in range(0, n_triples, chunk):
        c1 = min(n_triples, c0 + chunk)
        m = c1 - c0
        l2 = np.column_stack([la[c0:c1], lb[c0:c1]]).reshape(-1)
        xyz = np.zeros((m, 2, 3))
        xyz[:, 1] = B[c0:c1]
        mols = {"nshells": np.full(m, 2), "l": l2, "nprim": np.ones(2 * m, dtype=np.int32),
                "exps": np.column_stack([alpha[c0:c1], beta[c0:c1]]).reshape(-1), "coefs": np.ones(2 * m),
                "xyz": xyz.reshape(-1, 3)}
        Cd = torch.tensor(C[c0:c1], device=dev)
        Zd = torch.tensor(Z[c0:c1], device=dev)
        blocks = {}
        for name, prec in (("fp64", shgo.SHGO_PREC_FP64), ("bulk", shgo.SHGO_PREC_FP32_BULK),
                           ("plain", shgo.SHGO_PREC_FP32_PLAIN)):
            t0 = time.perf_counter()
            batch = shgo.Batch.from_arrays(mols, np.ones(m, dtype=np.int64), precision=prec)
            out = shgo.nuclear_attraction_batched(batch, Cd, Zd)
            torch.cuda.synchronize()
            t_gpu += time.perf_counter() - t0
            oh = out.cpu().numpy()
            per = {}
            for k in np.unique(cls[c0:c1]):
                i, j = int(k) // 9, int(k) % 9
                na, nb = 2 * i + 1, 2 * j + 1
                ms = np.nonzero(cls[c0:c1] == k)[0]
                idx = (batch.mol_off[ms][:, None, None] + np.arange(na)[None, :, None] * (na + nb) + na
                       + np.arange(nb)[None, None, :])
                per[int(k)] = (ms, oh[idx])
            blocks[name] = per
            batch.close()
            del out
        for k, (ms, v64) in blocks["fp64"].items():
            errs[k]["bulk"].append(rel(blocks["bulk"][k][1], v64, 1e-290))
            errs[k]["plain"].append(rel(blocks["plain"][k][1], v64, 1e-290))
            for t_local, blk in zip(ms, v64):
                t = c0 + int(t_local)
                if t in keep:
                    fp64_blocks[t] = blk
    res_f64 = [blk for part in job_f64.get() for blk in part]
    res_ext = [blk for part in job_ext.get() for blk in part]
    pool.close()
    pool.join()
    ref_f64 = dict(zip(ord_f64.tolist(), res_f64))
    ref_ext = dict(zip(ord_ext.tolist(), res_ext))

    def stat(v):
        v = np.concatenate(v) if isinstance(v, list) and v and isinstance(v[0], np.ndarray) else np.asarray(v)
        return {"max": float(v.max()), "median": float(np.median(v)), "n": int(v.size)} if v.size else None

    per_class, all_b, all_p, all_o, all_x = {}, [], [], [], []
    for k in range(81):
        i, j = k // 9, k % 9
        row = {"n": int(np.sum(cls == k)), "bulk_vs_fp64": stat(errs[k]["bulk"]),
               "plain_vs_fp64": stat(errs[k]["plain"])}
        skip = 1.01e-20 * 20.0  # below the primitive-pair bound the GPU path may skip by design
        eo, ex, od = [], [], []
        for t in sub_f64[k]:
            r, g = ref_f64[int(t)], fp64_blocks[int(t)]
            if np.max(np.abs(r)) > skip:
                eo.append(np.max(np.abs(g - r)) / np.max(np.abs(r)))
        for t in sub_ext[k]:
            r, g = ref_ext[int(t)], fp64_blocks[int(t)]
            if np.max(np.abs(r)) > skip:
                ex.append(np.max(np.abs(g - r)) / np.max(np.abs(r)))
                if int(t) in ref_f64:
                    od.append(np.max(np.abs(ref_f64[int(t)] - r)) / np.max(np.abs(r)))
        row["fp64_vs_oracle_double"] = stat(eo)
        row["fp64_vs_oracle_extended"] = stat(ex)
        row["oracle_double_vs_extended"] = stat(od)
        per_class[f"{i},{j}"] = row
        all_b += errs[k]["bulk"]
        all_p += errs[k]["plain"]
        all_o += eo
        all_x += ex
    line = {"precision_sweep": {
        "triples": n_triples, "oracle_double_per_class": n_oracle, "oracle_extended_per_class": n_ext,
        "oracle_extended_bits": oracle.real_bits("ld"), "host_cores": ncpu,
        "measure": "per (shell pair, nucleus) block: max|x - y| / max|y|; blocks with max|y| below 1e-290 "
                   "(K_AB underflow) or, against the oracle, below the primitive-pair bound left out",
        "fp32_bulk_vs_fp64": stat(all_b), "fp32_plain_vs_fp64": stat(all_p),
        "fp64_vs_oracle_double": stat(all_o), "fp64_vs_oracle_extended": stat(all_x),
        "gpu_s": t_gpu, "wall_s": time.perf_counter() - t_start, "per_class": per_class}}
    print(json.dumps(line), flush=True)
    return 0


def run_coulomb2c(args) -> int:
    """Two-centre Coulomb matrix (a|b) of the benchmark molecule's basis (32 atoms, one uncontracted shell per
    l = 0..6 per atom, 1568 functions): one step = the whole matrix.  Each shell pair is one block; the
    arithmetic per pair is small, so the kernel is rated against HBM for the matrix it writes."""
    import torch

    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W
    b, _, _ = W.config2()
    B = shgo.Basis(b)
    stream = torch.cuda.current_stream()
    out = torch.empty((B.nbf, B.nbf), dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda")  # 256 MiB, larger than L2
    for _ in range(max(3, args.warmup)):
        shgo.coulomb_2c(B, out=out, stream=stream)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 200))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        shgo.coulomb_2c(B, out=out, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs]))
    npairs = B.npairs
    written = float(B.nbf) * B.nbf * 8
    peaks = {}
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = written / (ms / 1e3) / 1e9
    line = {"metric": "two-centre Coulomb shell pairs/s", "value": npairs / (ms / 1e3), "unit": "shell-pairs/s",
            "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"(a|b) of the high-l benchmark basis: {len(b['l'])} shells, {B.nbf} functions",
                       "shell_pairs": npairs, "l2": "flushed between steps (256 MiB write, outside step events)"},
            "roofline": {"bound": "hbm", "kernel": "k_coulomb2c", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "note": "bytes of the matrix written (both triangles) per step; the inputs are a few KB",
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"}}
    print(json.dumps(line), flush=True)
    B.close()
    return 0


def _eri_pairs(basis):
    """Shell pairs as the library forms them: (l, nprim) of the pair with la >= lb, one per unordered pair."""
    ls, nps = [int(x) for x in basis["l"]], [int(x) for x in basis["nprim"]]
    out = []
    for la in range(9):
        A = [s for s in range(len(ls)) if ls[s] == la]
        for lb in range(la + 1):
            B = [s for s in range(len(ls)) if ls[s] == lb]
            for x, sa in enumerate(A):
                for sb in (B[:x + 1] if la == lb else B):
                    out.append((la, lb, nps[sa] * nps[sb]))
    return out


def eri_flops(basis) -> tuple[float, int]:
    """Algorithmic FP64 flops (FMA = 2) of the quartet kernels of one shgo_eri call, and the unique shell
    quartets.  Per primitive quartet: the radial factors Z (one FMA per Boys term of each (L, M, K) entry of
    Lambda_t = la + lb + lc + ld), the interaction matrix I (one FMA per Gaunt term of every bra x ket entry)
    and X += I D_cd^T (nr1 nr2 ncd FMAs); per bra primitive pair and ket pair D_ab X (nab ncd nr1 FMAs); the
    reduction over bra primitive pairs (nab ncd adds each).  The distributions (once per primitive pair) are
    not counted."""
    from paper_2404_16245_gb300 import shgo

    def n_r(lam):
        return (lam + 1) * (lam + 2) * (lam + 3) // 6

    gaunt_terms = {}

    def nterms(L1, M1, L2, M2):
        key = (L1, M1, L2, M2)
        if key not in gaunt_terms:
            n = 0
            for L in range(abs(L1 - L2), L1 + L2 + 1, 2):
                for M in {abs(M1) + abs(M2), -(abs(M1) + abs(M2)), abs(abs(M1) - abs(M2)), -abs(abs(M1) - abs(M2))}:
                    if abs(M) <= L and abs(shgo.host_gaunt(L1, M1, L2, M2, L, M)) > 1e-15:
                        n += 1
            gaunt_terms[key] = n
        return gaunt_terms[key]

    iterms = {}

    def i_terms(l1, l2):
        if (l1, l2) not in iterms:
            t = 0
            for L1 in range(l1 + 1):
                for L2 in range(l2 + 1):
                    w = ((l1 - L1) // 2 + 1) * ((l2 - L2) // 2 + 1)
                    t += w * sum(nterms(L1, M1, L2, M2) for M1 in range(-L1, L1 + 1) for M2 in range(-L2, L2 + 1))
            iterms[(l1, l2)] = t
        return iterms[(l1, l2)]

    def z_terms(lt):
        return sum((2 * L + 1) * sum(K + 1 for K in range((lt - L) // 2 + 1)) for L in range(lt + 1))

    pairs = _eri_pairs(basis)
    order = sorted(range(len(pairs)), key=lambda i: (pairs[i][0] * (pairs[i][0] + 1) // 2 + pairs[i][1]))
    pairs = [pairs[i] for i in order]
    flops, nq = 0.0, 0
    for i, (la, lb, np1) in enumerate(pairs):
        for (lc, ld, np2) in pairs[:i + 1]:
            l1, l2 = la + lb, lc + ld
            nab, ncd = (2 * la + 1) * (2 * lb + 1), (2 * lc + 1) * (2 * ld + 1)
            per_pq = 2 * (z_terms(l1 + l2) + i_terms(l1, l2) + n_r(l1) * n_r(l2) * ncd)
            flops += np1 * np2 * per_pq + np1 * 2 * nab * ncd * n_r(l1) + np1 * nab * ncd
            nq += 1
    return flops, nq


def run_eri(args) -> int:
    """Four-centre electron-repulsion integrals (ab|cd) of the plain FP64 basis (4 atoms in a 6 bohr cube,
    l = 0, 1, 2 shells of 3 primitives on every atom: 12 shells, 36 functions, 78 shell pairs, 3081 unique
    shell quartets): one step = the whole nbf^4 tensor.  Steps cycle over seeded replicas of that
    distribution, all resident on the device; L2 is flushed between steps (outside the step events)."""
    import torch

    import oracle
    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W

    stream = torch.cuda.current_stream()
    R = 4
    dicts = [W.config1(replica=r)[0] for r in range(R)]
    bases = [shgo.Basis(b) for b in dicts]
    n = bases[0].nbf
    outs = [torch.empty((n, n, n, n), dtype=torch.float64, device="cuda") for _ in range(R)]
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda")  # 256 MiB, larger than L2
    for k in range(max(3, args.warmup)):
        shgo.eri(bases[k % R], out=outs[k % R], stream=stream)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 200))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler(0)
    sampler.start()
    for k, (e0, e1) in enumerate(evs):
        flush.zero_()
        e0.record(stream)
        shgo.eri(bases[k % R], out=outs[k % R], stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs]))
    flops, nq = eri_flops(dicts[0])
    integrals = sum((2 * la + 1) * (2 * lb + 1) for la, lb, _ in _eri_pairs(dicts[0]))
    clk = clocks.get("sm_max_mhz") or 2070.0
    achieved = flops / (ms / 1e3) / 1e12
    pk64 = measure_fma_peak("fp64", stream)
    peak = pk64["tflops"]
    # end to end through the public API: basis from host arrays, the tensor back to pinned host memory
    host = torch.empty((n, n, n, n), dtype=torch.float64, pin_memory=True)
    h2d = sum(np.asarray(dicts[0][k]).nbytes for k in ("l", "nprim", "exps", "coefs", "xyz"))
    e2e_steps = 10
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        B = shgo.Basis(dicts[k % R])
        shgo.eri(B, out=outs[k % R], stream=stream)
        host.copy_(outs[k % R], non_blocking=True)
        torch.cuda.synchronize()
        B.close()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    # CPU oracle on the host cores, whole tensors of the same workload
    cpu = None
    if not args.no_cpu_baseline:
        oracle.build()
        cores = os.cpu_count() or 1
        done, t0 = 0, time.perf_counter()
        while True:
            oracle.eri(dicts[done % R], threads=cores)
            done += 1
            if time.perf_counter() - t0 >= min(args.cpu_seconds, 10.0):
                break
        el = time.perf_counter() - t0
        cpu = {"value": done * nq / el, "unit": "shell-quartets/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} whole tensors of the workload in {el:.1f} s"}
    # launches: distributions once per class, then part + reduce per class pair (one rectangle each here)
    ncls = len({(la, lb) for la, lb, _ in _eri_pairs(dicts[0])})
    launches = (ncls + 2 * ncls * (ncls + 1) // 2) * steps
    line = {"metric": "four-centre ERI unique shell quartets/s", "value": nq / (ms / 1e3), "unit": "shell-quartets/s",
            "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"(ab|cd) of the plain FP64 basis: 4 atoms, l = 0..2 x 3 primitives, {n} functions",
                       "unique_shell_quartets": nq, "unique_integrals_per_s": integrals * (integrals + 1) / 2 / (ms / 1e3),
                       "l2": "flushed between steps (256 MiB write, outside step events)"},
            "roofline": {"bound": "alu", "kernel": "k_eri_part", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "note": "algorithmic flops of k_eri_part + k_eri_reduce (model in bench.py) over the whole call",
                         "peak_source": "measured in this run: shgo_measure_fma_rate FP64, best of 3",
                         "peak_derived_nominal": fp64_peak_tflops(clk)},
            "cpu_baseline": cpu,
            "e2e": {"value": nq / e2e_s, "unit": "shell-quartets/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(n ** 4 * 8), "steps": e2e_steps,
                    "note": "basis upload + eri + D2H of the nbf^4 tensor, wall clock"},
            "clocks": clocks, "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    for B in bases:
        B.close()
    return 0


def run_peaks(args) -> int:
    """The roofline denominators of this GPU: FP64 (DFMA) and FP32 (FFMA) multiply-add rates from
    shgo_measure_fma_rate (2048 threads per SM, eight independent chains each, CUDA events), five
    launches each with the SM clock sampled during them, as one JSON line."""
    import torch
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    r64 = measure_fma_peak("fp64", stream, repeats=5)
    r32 = measure_fma_peak("fp32", stream, repeats=5)
    # launch-shape sweep: the rate should not depend on chains or threads once the pipe is full
    from paper_2404_16245_gb300 import shgo
    sweep = {}
    for name, prec, iters in (("fp64", shgo.SHGO_PREC_FP64, PEAK_ITERS["fp64"]),
                              ("fp32", shgo.SHGO_PREC_FP32_BULK, PEAK_ITERS["fp32"])):
        rows = []
        for chains in (4, 8, 16):
            for tps in (512, 1024, 2048):
                it = max(1, iters * 8 * 2048 // (chains * tps))
                rate, ms = shgo.shgo_measure_fma_rate_shape(prec, it, chains, tps, stream)
                rows.append({"chains": chains, "threads_per_sm": tps, "tflops": rate / 1e12, "ms": ms})
        sweep[name] = rows
    time.sleep(0.3)
    clocks = sampler.stop()
    clk = clocks.get("sm_max_mhz") or 2070.0
    line = {"workload": "peaks", "fp64_tflops": r64["tflops"], "fp32_tflops": r32["tflops"],
            "fp64_runs": r64, "fp32_runs": r32, "shape_sweep": sweep, "clocks": clocks,
            "fp64_nominal_at_max_clock": fp64_peak_tflops(clk), "fp32_nominal_at_max_clock": 2 * fp32_lane_peak_t(clk),
            "how": "shgo_measure_fma_rate: grid of 2048 threads per SM, each 8 independent FMA chains x 4 x iters; "
                   "best of 5 timed launches (CUDA events), one warm-up launch before each"}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(precision: str = "fp64", case: str = "highl") -> int:
    """Small fixed case for ncu captures: one warm and one measured V of the benchmark workload
    (highl) or of the first molecule of the batched workload (batched), or of the benchmark workload's
    derivative integrals (deriv) or field integrals (field) or overlap matrix (overlap); or the potential of a
    seeded density at 4096 points around it (esp; the gradient at the same points: espgrad); or 16 replicas of
    the benchmark molecule in one batch with each class's two kernels timed one after another, twice
    (replicas16)."""
    import torch

    from paper_2404_16245_gb300 import shgo
    from paper_2404_16245_gb300 import workloads as W
    if case == "replicas16":
        # 16 replicas of the benchmark molecule in one batch, each class's kernels timed one after another
        rb = [W.config2(replica=100 + k) for k in range(16)]
        batch = shgo.Batch([(bb, len(ZZ)) for bb, _, ZZ in rb])
        Cb = torch.tensor(np.concatenate([CC for _, CC, _ in rb]), device="cuda")
        Zb = torch.tensor(np.concatenate([ZZ for _, _, ZZ in rb]), device="cuda")
        outb = torch.empty(batch.out_size, dtype=torch.float64, device="cuda")
        for _ in range(2):
            shgo.shgo_nuclear_attraction_class_timed(batch.handle, Cb.shape[0], Cb.data_ptr(), Zb.data_ptr(),
                                                     outb.data_ptr(), None)
        torch.cuda.synchronize()
        print("profile case ok", batch.out_size)
        batch.close()
        return 0
    if case == "batched":
        b, C, Z = W.config3_molecule(np.random.Generator(np.random.PCG64(3000)))
    else:
        b, C, Z = W.config2()
    B = shgo.Basis(b, precision={"fp64": shgo.SHGO_PREC_FP64, "fp32": shgo.SHGO_PREC_FP32_BULK}[precision])
    Cd = torch.tensor(C, device="cuda")
    Zd = torch.tensor(Z, device="cuda")
    if case in ("esp", "espgrad"):
        rng = np.random.default_rng(7000)
        d = rng.normal(size=(B.nbf, B.nbf))
        D = torch.tensor((d + d.T) / 2, device="cuda")
        X = torch.tensor(rng.uniform(-4.0, 24.0, (4096, 3)), device="cuda")
        for _ in range(2):
            V = shgo.esp(B, D, X) if case == "esp" else shgo.esp_gradient(B, D, X)
        torch.cuda.synchronize()
        print("profile case ok", tuple(V.shape))
        B.close()
        return 0
    for _ in range(2):
        if case == "overlap":
            V = shgo.overlap(B)
        elif case == "deriv":
            V = shgo.nuclear_attraction_deriv(B, Cd, Zd)
        elif case == "field":
            V = shgo.nuclear_field(B, Cd, Zd)
        else:
            V = shgo.nuclear_attraction(B, Cd, Zd)
    torch.cuda.synchronize()
    print("profile case ok", tuple(V.shape))
    B.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-case", nargs="?", const="highl", choices=["highl", "batched", "deriv", "field", "replicas16",
                                                                     "esp", "espgrad", "overlap"],
                    help="one warm + one measured call, for ncu (the benchmark molecule or one batched molecule)")
    ap.add_argument("--precision-sweep", type=int, default=0, metavar="N",
                    help="per-class FP32-bulk / FP32-plain / FP64 error study on N random triples")
    ap.add_argument("--sweep-oracle", type=int, default=200,
                    help="triples per (la, lb) class also checked against the double oracle")
    ap.add_argument("--sweep-ext", type=int, default=20,
                    help="triples per (la, lb) class also checked against the extended-precision oracle")
    ap.add_argument("--workload", default="highl", choices=["highl", "batched", "screened", "esp", "coulomb2c", "eri", "peaks",
                                                          "deriv", "shard", "overlap"],
                    help="highl = the 32-atom l <= 6 molecule (default); batched = many contracted molecules")
    ap.add_argument("--molecules", type=int, default=64, help="molecules of the batched workload")
    ap.add_argument("--points", type=int, default=100000, help="points of the potential workload")
    ap.add_argument("--atoms", type=int, default=200, help="atoms of the screening cluster")
    ap.add_argument("--train-atoms", type=int, default=200,
                    help="atoms of the training cluster (as large as the evaluation cluster: the network "
                         "under-predicts outside the distances it was trained on)")
    ap.add_argument("--train-triples", type=int, default=1_000_000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--target-error", type=float, default=1e-10,
                    help="screening: largest error allowed on any V element (shared by the nuclei of a pair)")
    ap.add_argument("--threshold", type=float, default=0.0,
                    help="screening: per-triple threshold (0 = target error / number of nuclei)")
    ap.add_argument("--margin", type=float, default=0.0,
                    help="screening: safety factor below the threshold (0 = calibrated on held-out triples)")
    ap.add_argument("--audit", type=float, default=0.01, help="fraction of skipped triples checked exactly")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="shgo", choices=["shgo", "reference"])
    ap.add_argument("--replicas", type=int, default=8)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="fp32 = FP32-bulk nucleus loop (FP64 Boys, coupling and translation)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-class-batch", action="store_true", help="skip the 64-replica per-class timing")
    ap.add_argument("--speedup-molecules", type=int, default=16,
                    help="molecules of the batched workload for the speed-up at 1e-10 in the default line (0 = skip)")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args.precision, args.profile_case)
    if args.precision_sweep:
        return run_precision_sweep(args.precision_sweep, args.sweep_oracle, args.sweep_ext)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "screened":
        return run_screened(args)
    if args.workload == "esp":
        return run_esp(args)
    if args.workload == "deriv":
        return run_deriv(args)
    if args.workload == "coulomb2c":
        return run_coulomb2c(args)
    if args.workload == "overlap":
        return run_overlap(args)
    if args.workload == "eri":
        return run_eri(args)
    if args.workload == "peaks":
        return run_peaks(args)
    ws, rank, local = _dist()
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            return run_reference(args, ws, rank)
        if args.workload == "shard":
            return run_shard(args, ws, rank, local)
        return run_shgo(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
