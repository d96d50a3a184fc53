#!/usr/bin/env python3
"""Benchmark: g g -> t t~ g g matrix elements per second on one GB300.

Workload (the paper's headline process, Tables 1-2): 524288 RAMBO events at
sqrt(s) = 1.5 TeV, Philox seed 3, mt = 173 GeV, Gamma_t = 1.4915 GeV,
alpha_s = 0.118.  A step is one mg_sigma call over the whole batch (steps
A1-A6: momentum staging, wavefunctions, diagrams, colour sum, helicity sum),
with the good-helicity set-up (A0) done once before timing.  The headline
value is the mixed-precision path; the FP64 path on the same events, the
mixed-vs-FP64 accuracy, an end-to-end number through host buffers, the
roofline of the dominant kernel and the FP64 CPU oracle's throughput on a
bounded sample are reported beside it, with the other workloads of the set
(e+e- -> mu+mu-, g g -> t t~, g g -> t t~ g g g: mixed and FP64 throughput,
each kernel's roofline fraction, accuracy against the oracle) under
"configs", and a run of the continuous-batching request loop (Poisson
arrivals, four processes, p50/p99 latency; 2000 mixed and 200 FP64 requests,
then the first half / quarter of them again at 70 % load; --serve: twice as
many).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

Multi-GPU (torchrun): events are independent, so each rank evaluates its own
batch (event offsets rank * nevt) with no data-path collective: weak scaling.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PROC = "g g > t t~ g g"
SQRTS = 1500.0
SEED = 3
NEVT = 524288
# the other configurations of the workload set (--proc): process, sqrt(s), seed, events
WORKLOADS = {
    "eemumu": ("e+ e- > mu+ mu-", 500.0, 1, 16384),
    "ggtt": ("g g > t t~", 1000.0, 2, 524288),
    "ggttgg": ("g g > t t~ g g", 1500.0, 3, 524288),
    "ggttggg": ("g g > t t~ g g g", 2000.0, 4, 65536),
    "uutt": ("u u~ > t t~", 1000.0, 7, 524288),
    "uuttg": ("u u~ > t t~ g", 1200.0, 8, 524288),
    "uuttgg": ("u u~ > t t~ g g", 1500.0, 9, 524288),
}
METRIC = "gg→tt̄gg MEs/s on 1 GB300, FP64 vs mixed (≤1e-5 rel err); serve p50/p99 ms"
L2_FLUSH_BYTES = 256 << 20
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the mixed
# kernel from one ncu capture (sigma_tc_kernel of g g -> t t~ g g, mixed,
# 65536 events, one launch): workload -> (events captured, bytes, digest of
# the kernel sources at capture time); scaled to a launch by its events (the
# traffic is per event: momenta in, |M|^2 out).  Reported as null once the
# sources differ from the captured ones (kernel_digest()).
NCU_TRAFFIC = {"ggttgg": (65536, 12815104 + 745216, "bd63ce2f23a8d439")}
KERNEL_SOURCES = ("mg_kernels.cuh", "mg_vertices.cuh", "mg_colour_tc.cuh", "mg_flowstore.cuh")

SERVE_PROCS = {  # process -> sqrt(s)
    "e+ e- > mu+ mu-": 500.0,
    "g g > t t~": 1000.0,
    "g g > t t~ g g": 1500.0,
    "g g > t t~ g g g": 2000.0,
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during timing."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_digest(tag: str) -> str:
    """sha256 (16 hex digits) of the hand-written kernel sources and of the
    process's flop count (which changes with its generated code)."""
    import hashlib
    d = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2303_18244_gb300", "csrc", f), "rb") as fh:
            d.update(fh.read())
    d.update(json.dumps(load_flops(tag), sort_keys=True).encode())
    return d.hexdigest()[:16]


def traffic_per_launch(tag: str, nevt: int):
    cap = NCU_TRAFFIC.get(tag)
    if cap is None or cap[2] != kernel_digest(tag):
        return None
    return cap[1] * nevt / cap[0]


def measured_peak(key: str):
    """A peak measured on this machine's GPUs (copy bandwidth GB/s, BF16 GEMM
    TFLOP/s), or None."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return None


def load_flops(tag: str) -> dict:
    with open(os.path.join(ROOT, "paper_2303_18244_gb300", "flops.json")) as f:
        return json.load(f)[tag]


def launches_per_sigma(proc: str, nevt: int, ngood: int) -> int:
    """Kernel launches of one mixed mg_sigma call: one, except for gg -> t t~ g g g,
    whose two-phase path launches the flow and colour kernels once per slice
    of the good helicities, the slices sized to a 1 GiB flow workspace
    (120 complex FP32 flows per helicity-event row, events padded to 128)."""
    if proc != "ggttggg":
        return 1
    per_hel = 120 * ((nevt + 127) // 128 * 128) * 8
    hs = max(1, min(ngood, (1 << 30) // per_hel))
    return 2 * ((ngood + hs - 1) // hs)


def time_oracle(proc: str, sqrts: float, seed: int, first_event: int, budget_s: float = 12.0,
                one_core: bool = True, max_events: int = 1 << 20):
    """FP64 oracle on the host cores over a bounded sample of the workload's
    first events (at most max_events, the workload's own size): (MEs/s, cores,
    n, seconds, MEs/s on one core, oracle values)."""
    import oracle as O
    from paper_2303_18244_gb300.inputs import process_momenta
    cores = os.cpu_count() or 1
    O.me(proc, process_momenta(proc, sqrts, cores, seed, first_event))  # colour matrix, warm
    n = min(cores, max_events)
    best = None
    while True:
        p = process_momenta(proc, sqrts, n, seed, first_event)
        t = time.perf_counter()
        ref = O.me(proc, p, threads=cores)
        dt = time.perf_counter() - t
        best = (n / dt, cores, n, dt)
        if dt >= budget_s / 4 or n >= max_events:
            break
        n = min(max_events, int(n * min(8.0, max(2.0, budget_s / 4 / max(dt, 1e-3)))))
    one = None
    if one_core:  # one core, on a sample about two seconds long
        n1 = max(1, min(n, int(best[0] / cores * 2.0)))
        t = time.perf_counter()
        O.me(proc, p[:n1], threads=1)
        one = n1 / (time.perf_counter() - t)
    return best + (one, ref)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2303_18244_gb300.inputs import process_momenta  # noqa: F401
    vals = []
    info = None
    for _ in range(args.warmup if args.warmup < 1 else 1):
        time_oracle(PROC, SQRTS, SEED, 0, budget_s=2.0, one_core=False, max_events=NEVT)
    for _ in range(args.steps):
        v, cores, n, dt, _, _ = time_oracle(PROC, SQRTS, SEED, 0, budget_s=8.0, one_core=False, max_events=NEVT)
        vals.append(v)
        info = (cores, n)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MEs/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * info[1] / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (RAMBO flat phase space, Philox seed 3)",
            "config": {"workload": f"{PROC}, {NEVT} events at sqrt(s)={SQRTS:.0f} GeV (sample of {info[1]})",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "MEs/s", "cores": info[0], "kind": "oracle",
                             "sample": f"{info[1]} events of the workload per step"},
            "e2e": {"value": v, "unit": "MEs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--proc", default="ggttgg", choices=sorted(WORKLOADS))
    ap.add_argument("--nevt", type=int, default=None)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--serve", action="store_true",
                    help="longer serving benchmark (4000 mixed and 400 FP64 requests instead of 2000 and 200)")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads of the set")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-requests", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    global PROC, SQRTS, SEED, NEVT
    PROC, SQRTS, SEED, NEVT = WORKLOADS[args.proc]
    if args.nevt is None:
        args.nevt = NEVT
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2303_18244_gb300 import mg
    from paper_2303_18244_gb300.inputs import process_momenta
    from paper_2303_18244_gb300.shard import barrier, event_block, max_over_ranks

    first, nevt = event_block(rank, world, args.nevt)
    p = process_momenta(PROC, SQRTS, nevt, SEED, first_event=first)
    calib = process_momenta(PROC, SQRTS, 1024, SEED + 1000)
    mom = torch.from_numpy(p).cuda()
    out = torch.empty(nevt, dtype=torch.float64, device="cuda")
    out64 = torch.empty(nevt, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    hmix = mg.Process(PROC, precision=mg.MG_MIXED)
    h64 = mg.Process(PROC, precision=mg.MG_FP64)
    ngood, _ = mg.good_helicities(hmix, torch.from_numpy(calib).cuda())
    mg.good_helicities(h64, torch.from_numpy(calib).cuda())

    def timed_call(fn, steps, warmup):
        """CUDA-event times (ms) of fn() on the stream, L2 flushed before each."""
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        per = []
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps (inputs are smaller than L2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            per.append((e0, e1))
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in per]
        barrier()
        return ms

    def timed(h, o, steps, warmup):
        return timed_call(lambda: mg.sigma(h, mom, o, stream), steps, warmup)

    clocks = ClockSampler(local)
    clocks.start()
    ms_mix = timed(hmix, out, args.steps, args.warmup)
    clk = clocks.stop()
    assert mg.process_status(hmix) == 0
    ms_64 = timed(h64, out64, args.fp64_steps, 1)
    assert mg.process_status(h64) == 0
    # the paper's own mixed mode (FP64 diagrams, FP32 colour algebra) for comparison
    hpap = mg.Process(PROC, precision=mg.MG_MIXED_PAPER)
    mg.good_helicities(hpap, torch.from_numpy(calib).cuda())
    outp = torch.empty(nevt, dtype=torch.float64, device="cuda")
    ms_pap = timed(hpap, outp, 1, 1)
    assert mg.process_status(hpap) == 0
    # the paper's float mode (every step in FP32)
    hflt = mg.Process(PROC, precision=mg.MG_FLOAT)
    mg.good_helicities(hflt, torch.from_numpy(calib).cuda())
    outf = torch.empty(nevt, dtype=torch.float64, device="cuda")
    ms_flt = timed(hflt, outf, 1, 1)
    assert mg.process_status(hflt) == 0

    t_mix, t_64, t_pap, t_flt = max_over_ranks([sum(ms_mix), sum(ms_64) / len(ms_64), sum(ms_pap), sum(ms_flt)],
                                               device="cuda")
    value = world * nevt * args.steps / (t_mix * 1e-3)
    value64 = world * nevt / (t_64 * 1e-3)

    # accuracy of the mixed path against the FP64 GPU path (itself held to the
    # FP64 oracle at <= 1e-12 by the parity tests) on every event of the batch
    a = out.cpu().numpy()
    b = out64.cpu().numpy()
    rel = np.abs(a - b) / np.abs(b)
    rel_f = np.abs(outf.cpu().numpy() - b) / np.abs(b)

    # end to end through the C ABI from pinned host buffers
    hp = torch.from_numpy(p).pin_memory()
    ho = torch.empty(nevt, dtype=torch.float64).pin_memory()
    for _ in range(2):
        mg.sigma_host(hmix, hp, ho, stream)
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()  # same L2 state as the device-timed steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mg.sigma_host(hmix, hp, ho, stream)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_t = max_over_ranks([statistics.median(e2e_ms)], device="cuda")[0]

    # the same with the phase-space points generated on the device (mg_rambo,
    # the paper's proposed offload of the random-number -> momenta step):
    # only the MEs cross to the host
    dmom = torch.empty_like(mom)
    for _ in range(2):
        mg.rambo(hmix, SQRTS, SEED, first, dmom, stream)
        mg.sigma(hmix, dmom, out, stream)
    torch.cuda.synchronize()
    dev_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mg.rambo(hmix, SQRTS, SEED, first, dmom, stream)
        mg.sigma(hmix, dmom, out, stream)
        ho.copy_(out)  # D2H of the MEs (synchronous)
        dev_ms.append((time.perf_counter() - t0) * 1e3)
    dev_t = max_over_ranks([statistics.median(dev_ms)], device="cuda")[0]

    # the ME with the event-by-event choice of a good helicity and a colour
    # flow (mg_sigma_select, mixed: colour sum on CUDA cores), on the same events
    from paper_2303_18244_gb300.inputs import uniforms
    rnd = torch.from_numpy(np.ascontiguousarray(uniforms(SEED + 2000, first, nevt, 1)[:, 0, :2])).cuda()
    hel_o = torch.empty(nevt, dtype=torch.int32, device="cuda")
    col_o = torch.empty(nevt, dtype=torch.int32, device="cuda")
    out_s = torch.empty(nevt, dtype=torch.float64, device="cuda")
    ms_sel = timed_call(lambda: mg.sigma_select(hmix, mom, rnd, out_s, hel_o, col_o, None, stream), 2, 1)
    assert mg.process_status(hmix) == 0
    t_sel = max_over_ranks([statistics.median(ms_sel)], device="cuda")[0]

    # hit-or-miss unweighting (mg_unweight) of the workload's MEs, and of
    # 128 copies of them (67 M events, 1 GiB of weights and uniforms: HBM-bound)
    def unweight_ms(w, r):
        idx = torch.empty(w.shape[0], dtype=torch.int64, device="cuda")
        nacc = torch.empty(1, dtype=torch.int64, device="cuda")
        wmax = float(w.max())
        ms_u = timed_call(lambda: mg.unweight(w, r, wmax, idx, nacc, stream), 3, 2)
        return statistics.median(ms_u), int(nacc.item())
    r_u = rnd[:, 0].contiguous()
    uw_ms, uw_kept = unweight_ms(out, r_u)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(SEED + 3000)
    w_big = out.repeat(128)
    r_big = torch.rand(w_big.shape[0], dtype=torch.float64, device="cuda", generator=gen)
    uwb_ms, uwb_kept = unweight_ms(w_big, r_big)
    del w_big, r_big
    uw_t, uwb_t = max_over_ranks([uw_ms, uwb_ms], device="cuda")
    hbm_peak = measured_peak("hbm_gbs")
    # algorithmic bytes: w and r read once (16 B per event), 8 B per kept index
    uwb_bytes = 16 * 128 * nevt + 8 * uwb_kept

    fl = load_flops(args.proc)
    flops_evt = ngood * (fl["amp_flops_per_hel"] + fl["colour_dense_flops_per_hel"])
    kernel_ms = t_mix / args.steps
    achieved = flops_evt * nevt / (kernel_ms * 1e-3) / 1e12
    peak32 = mg.diag_fma_peak(0) / 1e3
    peak64 = mg.diag_fma_peak(1) / 1e3
    achieved64 = flops_evt * nevt / (t_64 * 1e-3) / 1e12

    traffic = traffic_per_launch(args.proc, nevt)

    res = {
        "metric": METRIC, "value": value, "unit": "MEs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_mix / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 denominators and helicity sum)",
        "data": "synthetic (RAMBO flat phase space, Philox seed 3)",
        "config": {"workload": f"{PROC}, {nevt} events/GPU at sqrt(s)={SQRTS:.0f} GeV, mixed precision",
                   "good_helicities": ngood, "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"events sharded, {world} rank(s), no collective"},
        "fp64": {"value": value64, "unit": "MEs/s", "ms_per_step": t_64,
                 "roofline": {"bound": "alu", "achieved": achieved64, "peak": peak64, "unit": "TFLOP/s",
                              "frac": achieved64 / peak64, "peak_source": "measured FP64 FMA loop (mg_diag)"}},
        "paper_mixed": {"value": world * nevt / (t_pap * 1e-3), "unit": "MEs/s",
                        "what": "FP64 diagrams + FP32 colour algebra (the paper's mixed mode)"},
        "float": {"value": world * nevt / (t_flt * 1e-3), "unit": "MEs/s",
                  "what": "every step in FP32 (the paper's float mode)",
                  "accuracy_vs_fp64": {"median": float(np.median(rel_f)), "p99": float(np.quantile(rel_f, 0.99)),
                                       "max": float(rel_f.max())}},
        "accuracy_mixed_vs_fp64": {"median": float(np.median(rel)), "p99": float(np.quantile(rel, 0.99)),
                                   "max": float(rel.max()), "events": nevt},
        "e2e": {"value": world * nevt / (e2e_t * 1e-3), "unit": "MEs/s",
                "h2d_bytes_per_step": int(p.nbytes), "d2h_bytes_per_step": int(nevt * 8)},
        "e2e_device_phase_space": {"value": world * nevt / (dev_t * 1e-3), "unit": "MEs/s",
                                   "what": "mg_rambo + mg_sigma + D2H of the MEs per step",
                                   "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(nevt * 8)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak32, "unit": "TFLOP/s",
                     "frac": achieved / peak32, "traffic": traffic,
                     "kernel": f"sigma kernel of {args.proc}, mixed",
                     "flops_per_event": flops_evt,
                     "peak_source": "measured FP32 FMA loop (mg_diag), burst"},
        "select": {"value": world * nevt / (t_sel * 1e-3), "unit": "MEs/s",
                   "what": "mg_sigma_select, mixed: the ME plus a good helicity and a colour flow per event "
                           "(colour sum on CUDA cores)"},
        "unweight": {"value": world * nevt / (uw_t * 1e-3), "unit": "events/s", "ms": uw_t, "kept": uw_kept,
                     "what": "mg_unweight of the workload's MEs (hit-or-miss, kept indices in order)",
                     "large": {"events": 128 * nevt, "ms": uwb_t, "kept": uwb_kept,
                               "roofline": {"bound": "hbm", "achieved": uwb_bytes / (uwb_t * 1e-3) / 1e9,
                                            "peak": hbm_peak, "unit": "GB/s",
                                            "frac": (uwb_bytes / (uwb_t * 1e-3) / 1e9) / hbm_peak
                                            if hbm_peak else None,
                                            "bytes_per_event": "16 read (w, r) + 8 per kept index",
                                            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)"}}},
        "gpu_launches": args.steps * launches_per_sigma(args.proc, nevt, ngood),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, n, dt, one, ref = time_oracle(PROC, SQRTS, SEED, first, max_events=nevt)
        res["cpu_baseline"] = {"value": v, "unit": "MEs/s", "cores": cores, "kind": "oracle",
                               "sample": f"the first {n} events of the workload ({dt:.1f} s wall)",
                               "value_one_core": one}
        # per-event relative error of both GPU paths against the oracle on that sample
        acc = {}
        for name, o in (("fp64", out64), ("mixed", out)):
            got = o[:n].cpu().numpy()
            r = np.abs(got - ref) / np.abs(ref)
            acc[name] = {"median": float(np.median(r)), "p99": float(np.quantile(r, 0.99)),
                         "max": float(r.max()), "events": int(n)}
            if name == "fp64":
                # where the FP64 oracle and the FP64 path differ by more than
                # 1e-12, the oracle's long-double build decides
                import oracle as O
                bad = np.nonzero(r > 1e-12)[0]
                r_adj = r.copy()
                if bad.size:
                    pb = process_momenta(PROC, SQRTS, n, SEED, first_event=first)[bad]
                    ext = O.me(PROC, pb, extended=True)
                    r_adj[bad] = np.abs(got[bad] - ext) / np.abs(ext)
                acc[name]["beyond_1e-12"] = int(bad.size)
                acc[name]["max_adjudicated"] = float(r_adj.max())
        res["accuracy_vs_oracle"] = acc
    if not args.no_configs and args.proc == "ggttgg" and world == 1:  # one GPU: the set's other workloads
        res["configs"] = {t: measure_config(t, mg, process_momenta, timed_call, peak32, peak64)
                          for t in ("eemumu", "ggtt", "ggttggg", "uuttgg")}
    if not args.no_serve and args.proc == "ggttgg":
        nreq = args.serve_requests or (4000 if args.serve else 2000)
        plan = {"mixed": nreq, "fp64": max(1, nreq // 10)}
        paced = {"mixed": max(1, nreq // 2), "fp64": max(1, nreq // 40)}
        res["serve"] = serve_bench(plan, mg, process_momenta, paced)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure_config(tag, mg, process_momenta, timed_call, peak32, peak64, oracle_budget_s=3.0):
    """One workload of the set, mixed and FP64: MEs/s from CUDA-event-timed
    steps (median of 3 after warm-up, L2 flushed before each), the roofline
    fraction of its kernels, and the per-event error of both paths against the
    oracle on the workload's first events (as many as the oracle evaluates in
    about oracle_budget_s on the host cores)."""
    import torch
    proc, sqrts, seed, nevt = WORKLOADS[tag]
    p = process_momenta(proc, sqrts, nevt, seed)
    mom = torch.from_numpy(p).cuda()
    calib = torch.from_numpy(process_momenta(proc, sqrts, 1024, seed + 1000)).cuda()
    fl = load_flops(tag)
    res = {"workload": f"{proc}, {nevt} events at sqrt(s)={sqrts:.0f} GeV, seed {seed}"}
    outs = {}
    for name, prec, warm in (("mixed", mg.MG_MIXED, 3), ("fp64", mg.MG_FP64, 1)):
        h = mg.Process(proc, precision=prec)
        ngood, _ = mg.good_helicities(h, calib)
        out = torch.empty(nevt, dtype=torch.float64, device="cuda")
        ms = timed_call(lambda: mg.sigma(h, mom, out), 3, warm)
        assert mg.process_status(h) == 0
        t = statistics.median(ms)
        flops = ngood * (fl["amp_flops_per_hel"] + fl["colour_dense_flops_per_hel"]) * nevt
        peak = peak32 if name == "mixed" else peak64
        r = {"value": nevt / (t * 1e-3), "unit": "MEs/s", "ms_per_step": t, "steps": len(ms),
             "good_helicities": ngood,
             "roofline": {"bound": "alu", "achieved": flops / (t * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                          "frac": flops / (t * 1e-3) / 1e12 / peak,
                          "peak_source": f"measured {'FP32' if name == 'mixed' else 'FP64'} FMA loop (mg_diag)"}}
        if name == "mixed" and tag == "ggttggg":
            r["kernels"] = two_phase_rooflines(h, mom, out, mg, fl, ngood, nevt)
        res[name] = r
        outs[name] = out.cpu().numpy()
        h.close()
    res["mixed_over_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    # accuracy against the oracle on the first events
    _, cores, n, dt, _, ref = time_oracle(proc, sqrts, seed, 0, budget_s=oracle_budget_s, one_core=False,
                                          max_events=nevt)
    acc = {"events": int(n), "sample": f"the first {n} events ({dt:.1f} s of the oracle on {cores} cores)"}
    for name in ("fp64", "mixed"):
        got = outs[name][:n]
        r = np.abs(got - ref) / np.abs(ref)
        acc[name] = {"median": float(np.median(r)), "p99": float(np.quantile(r, 0.99)), "max": float(r.max())}
        if name == "fp64":
            import oracle as O
            bad = np.nonzero(r > 1e-12)[0]
            if bad.size:
                ext = O.me(proc, p[:n][bad], extended=True)
                r = r.copy()
                r[bad] = np.abs(got[bad] - ext) / np.abs(ext)
            acc[name]["beyond_1e-12"] = int(bad.size)
            acc[name]["max_adjudicated"] = float(r.max())
    res["accuracy_vs_oracle"] = acc
    return res


def two_phase_rooflines(h, mom, out, mg, fl, ngood, nevt):
    """The two kernels of the two-phase mixed g g -> t t~ g g g call timed one
    by one (CUDA events between the launches, mg_diag_sigma_phases; median of
    3 calls): the flow kernel against the FP32 FMA peak (amplitude flops), the
    tensor-core colour kernel against HBM (it reads every helicity-event row
    of 120 complex FP32 flows once: 960 B per row) and, beside it, its
    tensor-pipe fraction (4 * 120^2 flop per row, the dense quadratic form)
    against the FP16 tcgen05 MMA rate measured by mg_diag_mma_peak (the
    measured BF16 GEMM peak beside it)."""
    runs = [mg.diag_sigma_phases(h, mom, out) for _ in range(3)]
    t1 = statistics.median(r[0] for r in runs)
    t2 = statistics.median(r[1] for r in runs)
    slices = runs[0][2]
    rows = ngood * ((nevt + 127) // 128 * 128)
    peak32 = mg.diag_fma_peak(0) / 1e3
    hbm = measured_peak("hbm_gbs")
    bf16 = measured_peak("bf16_tflops")
    fp16_mma = mg.diag_mma_peak()
    f1 = ngood * fl["amp_flops_per_hel"] * nevt / (t1 * 1e-3) / 1e12
    b2 = rows * 120 * 8 / (t2 * 1e-3) / 1e9
    f2 = 4 * 120 ** 2 * ngood * nevt / (t2 * 1e-3) / 1e12
    return {
        "slices": slices,
        "flows_tmem_kernel": {"ms": t1, "bound": "alu", "achieved": f1, "peak": peak32, "unit": "TFLOP/s",
                              "frac": f1 / peak32, "peak_source": "measured FP32 FMA loop (mg_diag)"},
        "colour_rows_tc_kernel": {"ms": t2, "bound": "hbm", "achieved": b2, "peak": hbm, "unit": "GB/s",
                                  "frac": b2 / hbm if hbm else None,
                                  "bytes_per_row": "960 (120 complex FP32 flows read once)",
                                  "peak_source": "measured copy bandwidth (hbm_gbs)",
                                  "tensor": {"achieved": f2, "peak": fp16_mma, "unit": "TFLOP/s",
                                             "frac": f2 / fp16_mma,
                                             "flop_per_row": "4 * 120^2",
                                             "peak_source": "measured FP16 tcgen05 MMA loop (mg_diag_mma_peak)",
                                             "bf16_gemm_peak": bf16}},
    }


def serve_run(srv, handles, reqs, gap_scale=1.0):
    """Submit reqs (process, events, gap s, momenta, output) at their Poisson
    gaps times gap_scale, wait for every result; latency = submit -> done."""
    ids = []
    t0 = time.perf_counter()
    t_next = t0
    for proc, n, gap, mom, me in reqs:
        t_next += gap * gap_scale
        while time.perf_counter() < t_next:
            pass
        ids.append(srv.submit(handles[proc], mom, me))
    lat, tot = [], 0
    for rid, (proc, n, *_rest) in zip(ids, reqs):
        while True:
            rc, st = srv.poll(rid, 1000000)
            if rc == 0:
                break
        lat.append(st.latency_us / 1e3)
        tot += n
    wall = time.perf_counter() - t0
    window = gap_scale * sum(r[2] for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "MEs_per_s": tot / wall, "requests": len(reqs), "events": tot,
            "mean_gap_ms": 1e3 * window / len(reqs), "offered_MEs_per_s": tot / window, "wall_s": wall}


def serve_bench(plan, mg, process_momenta, paced=None, utilisation=0.7):
    """Poisson arrivals (mean gap 2 ms) of requests drawn uniformly from four
    processes, log-uniform 256..65536 events each (Philox seed 5 drives the
    choices), served by the continuous-batching loop; p50/p99 latency.
    plan: precision name -> number of requests.  The workload offers several
    times the events per second one GPU evaluates (its gg -> t t~ g g g
    requests alone), so its latency is mostly time in the queue; with paced
    (precision name -> number of requests) the first requests are served again
    with every gap stretched so that the offered rate is `utilisation` times
    the rate the first run achieved: the latency of a loop that keeps up."""
    from paper_2303_18244_gb300.inputs import uniforms
    import torch
    out = {}
    for prec_name, prec in (("mixed", mg.MG_MIXED), ("fp64", mg.MG_FP64)):
        if prec_name not in plan:
            continue
        nreq = plan[prec_name]
        handles = {p: mg.Process(p, precision=prec) for p in SERVE_PROCS}
        for p, hh in handles.items():
            calib = process_momenta(p, SERVE_PROCS[p], 1024, 1005)
            mg.good_helicities(hh, torch.from_numpy(calib).cuda())
        u = uniforms(5, 0, nreq, 1)[:, 0, :]
        reqs = []
        for i in range(nreq):
            proc = list(SERVE_PROCS)[min(3, int(u[i, 0] * 4))]
            n = int(round(math.exp(math.log(256) + u[i, 1] * (math.log(65536) - math.log(256)))))
            gap = -2e-3 * math.log(u[i, 2])
            # the request's RAMBO events (seed 5, its own block of the stream),
            # generated on the device and handed to the client in host memory
            d = torch.empty((n, handles[proc].info.npar, 4), dtype=torch.float64, device="cuda")
            mg.rambo(handles[proc], SERVE_PROCS[proc], 5, i * 65536, d)
            reqs.append((proc, n, gap, d.cpu().numpy(), np.empty(n)))
        srv = mg.Server()
        r = serve_run(srv, handles, reqs)
        r["utilisation_offered"] = r["offered_MEs_per_s"] / r["MEs_per_s"]
        r["workload"] = ("Poisson arrivals (mean 2 ms), processes uniform over "
                         "ee->mumu/gg->tt~/gg->tt~gg/gg->tt~ggg, log-uniform 256-65536 events, seed 5")
        out[prec_name] = r
        if paced and prec_name in paced:
            sub = reqs[: paced[prec_name]]
            scale = r["utilisation_offered"] / utilisation
            rp = serve_run(srv, handles, sub, gap_scale=scale)
            rp["utilisation_target"] = utilisation
            rp["workload"] = (f"the first {len(sub)} requests of the same stream, every gap times {scale:.1f} "
                              f"(offered rate {utilisation} of the rate served above)")
            out[prec_name + "_paced"] = rp
        srv.close()
    return out


if __name__ == "__main__":
    sys.exit(main())
