"""Benchmark: sliced bucket-elimination amplitudes of a 7x7-grid random circuit
(depth 1+32+1) on GB300.

One step = one amplitude <x|C|0^49>: all 2^p slices (p chosen so every slice's
largest bucket has at most 2^28 entries) contracted through the C-ABI call
tnq_contract_sliced and summed in FP64. The JSON line reports
slice-contractions/s (the metric), time per amplitude, the relative error of
the amplitude (every slice recomputed by the FP64 oracle) and of its worst
slice, the roofline of the fused bucket kernel, and the oracle's own speed on
the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank contracts its own bitstring's amplitude (weak
scaling, no collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIGS = {
    # name: (rows, cols, cycles, max_bag_log2, min_p, max_p)
    "7x7_d1+32+1": (7, 7, 32, 28, 0, 40),
    "6x6_d1+24+1": (6, 6, 24, 24, 4, 8),
    "4x4_d1+16+1": (4, 4, 16, 0, 0, 0),
}
METRIC = "slice-contractions/s & time per amplitude, 7x7 d1+32+1; %roofline; err vs FP64"


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.samples = []  # (host time, csv line)
        self.t0 = self.t1 = None  # the timed region, set by the caller

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.samples.append((time.perf_counter(), line))

    def __enter__(self):
        import threading

        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        t = time.perf_counter()
        while not self.samples and time.perf_counter() - t < 3.0:  # sampling runs before timing starts
            time.sleep(0.02)
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)  # one more sample after the region
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.reader.join(timeout=5)
        return False

    def summary(self):
        """Median SM clock and throttle reasons of the samples taken inside the
        timed region (the nearest ones if the region was shorter than a sample)."""
        inside = [l for t, l in self.samples if self.t0 is not None and self.t0 <= t <= self.t1]
        lines = inside
        if not lines and self.samples and self.t0 is not None:
            mid = 0.5 * (self.t0 + self.t1)
            lines = [min(self.samples, key=lambda x: abs(x[0] - mid))[1]]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "samples_in_timed_region": len(inside)}


# ncu DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of every
# k_group launch of a one-slice batch of this workload (capture command in
# profiles/k_group_7x7_d1+32+1.md), valid only while the fused-chain kernel's
# source (runtime.cu between the "Fused chain of buckets" and "K4: amplitude"
# comments) hashes to `kernel_sha1` and the plan has the recorded tuning and
# k_group launch count (reported as null otherwise). Per launch at batch B:
# bytes_one_slice x B / k_group launches per batch (traffic scales with the
# slices of a batch; item-invariant operands are read once per batch, so this
# slightly overstates it).
MEASURED_TRAFFIC = {"k_group": [
    {"kernel_sha1": "9600051a4d6febd8fe8034590085acd1e4118364", "tuning": [4, 64], "bytes_one_slice": 106121216.0,
     "launches": 12,
     "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum -k regex:k_group -s 12 -c 12 on a one-slice "
                "batch of the tuned default plan (tuning 2^4 / 64)"},
]}


def kernel_source_sha1():
    """SHA-1 of the fused-chain kernel's source region of runtime.cu."""
    import hashlib

    with open(os.path.join(ROOT, "paper_2004_10892_gb300", "csrc", "runtime.cu")) as f:
        text = f.read()
    a = text.index("// Fused chain of buckets")
    b = text.index("// K4: amplitude")
    return hashlib.sha1(text[a:b].encode()).hexdigest()


# FP32 CUDA-core peak of GB300 from unit counts and clocks: 152 SMs x 128 FP32
# lanes x 2 flops (FMA) x 2.07 GHz (the maximum SM clock in MEASURED_PEAKS.json).
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(peaks):
    return 152 * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def measured_fp32_peak(L, stream):
    """FP32 FMA peak measured on this device (tnq_internal_fp32_peak: an FMA
    loop on every SM, best of 5 launches timed with CUDA events), TFLOP/s."""
    out = ctypes.c_double()
    L.tnq_internal_fp32_peak.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    if L.tnq_internal_fp32_peak(5, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out)) != 0:
        return None
    return out.value


def launch_roofline(L, plan, bits, ws, B, n_sl, stream, peaks, info):
    """Times every launch of one batch with CUDA events on the launching stream
    and returns the roofline of the kernel with the largest share of time."""
    import numpy as np

    nb = info["n_buckets"] + 64
    ms = (ctypes.c_float * nb)()
    by = (ctypes.c_double * nb)()
    fl = (ctypes.c_double * nb)()
    bag = (ctypes.c_int * nb)()
    kind = (ctypes.c_int * nb)()
    n_out, b_out = ctypes.c_int(), ctypes.c_int()
    P = ctypes.POINTER
    L.tnq_internal_profile.argtypes = [ctypes.c_void_p, P(ctypes.c_uint8), ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int,
                                       P(ctypes.c_float), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int),
                                       P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]
    bb = np.ascontiguousarray(np.array(bits, dtype=np.uint8))
    rc = L.tnq_internal_profile(plan.handle, bb.ctypes.data_as(P(ctypes.c_uint8)), 0, n_sl,
                                ctypes.c_void_p(ws.data_ptr()), ws.numel(), B, ctypes.c_void_p(stream.cuda_stream),
                                nb, ms, by, fl, bag, kind, ctypes.byref(n_out), ctypes.byref(b_out))
    if rc != 0:
        return None
    n = n_out.value
    grp = [i for i in range(n) if 0 < kind[i] < 100]
    one = [i for i in range(n) if kind[i] == 0]
    gem = [i for i in range(n) if kind[i] >= 100]
    t_grp = sum(ms[i] for i in grp)
    t_one = sum(ms[i] for i in one)
    t_gem = sum(ms[i] for i in gem)
    tot = t_grp + t_one + t_gem
    hbm = peaks["hbm_gbs"]
    fp32_meas = measured_fp32_peak(L, stream)
    fp32 = fp32_meas if fp32_meas else fp32_peak_tflops(peaks)
    fp32_src = ("measured: FFMA loop on every SM (tnq_internal_fp32_peak), best of 5 CUDA-event-timed launches; "
                f"derived 152 SMs x 128 lanes x 2 x max clock = {fp32_peak_tflops(peaks):.1f}") if fp32_meas else \
        "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"
    one_gbs = sum(by[i] for i in one) / (t_one / 1e3) / 1e9 if t_one > 0 else None
    grp_tfs = sum(fl[i] for i in grp) / (t_grp / 1e3) / 1e12 if t_grp > 0 else None
    k_bucket = {"kernel": "k_bucket", "bound": "hbm", "achieved": one_gbs, "peak": hbm, "unit": "GB/s",
                "frac": one_gbs / hbm if one_gbs else None, "launches": len(one), "time_share": t_one / tot,
                "bytes_per_launch": sum(by[i] for i in one) / max(len(one), 1),
                "ms_per_launch": t_one / max(len(one), 1),
                "note": "per-step profile: every single bucket timed as its own launch (the captured graph "
                        "runs the item-invariant gate-fed ones as one k_bucket_level launch per level)"}
    big1 = [i for i in one if by[i] >= 64e6]  # launches large enough to stream at HBM speed
    t_big1 = sum(ms[i] for i in big1)
    if big1 and t_big1 > 0:
        gbs = sum(by[i] for i in big1) / (t_big1 / 1e3) / 1e9
        k_bucket["launches_ge_64MB"] = {"launches": len(big1), "achieved": gbs, "frac": gbs / hbm,
                                        "share_of_k_bucket_time": t_big1 / t_one,
                                        "each": [{"bag": bag[i], "MB": round(by[i] / 1e6, 1), "ms": round(ms[i], 4),
                                                  "gbs": round(by[i] / (ms[i] / 1e3) / 1e9, 1)} for i in big1]}
    k_group = {"kernel": "k_group", "bound": "alu", "achieved": grp_tfs, "peak": fp32, "unit": "TFLOP/s",
               "frac": grp_tfs / fp32 if grp_tfs else None, "launches": len(grp), "time_share": t_grp / tot,
               "flops_per_launch": sum(fl[i] for i in grp) / max(len(grp), 1),
               "ms_per_launch": t_grp / max(len(grp), 1),
               "peak_source": fp32_src}
    dom, other = (k_group, k_bucket) if t_grp >= t_one else (k_bucket, k_group)
    out = dict(dom)
    out["traffic"] = None
    if dom["kernel"] == "k_group" and grp:
        big = max(grp, key=lambda i: ms[i])
        out["largest_launch"] = {"ms": ms[big], "flops": fl[big], "algorithmic_bytes": by[big],
                                 "achieved_tflops": fl[big] / (ms[big] / 1e3) / 1e12 if ms[big] > 0 else None}
        for mt in MEASURED_TRAFFIC["k_group"]:
            if (mt["kernel_sha1"] == kernel_source_sha1() and mt["tuning"] == list(plan.tuning())
                    and mt["launches"] == len(grp) and mt["bytes_one_slice"] > 0):
                out["traffic"] = mt["bytes_one_slice"] * b_out.value / len(grp)
                out["traffic_source"] = mt["capture"] + ", x batch / k_group launches per batch"
    out["peak_source"] = dom.get("peak_source", "measured (MEASURED_PEAKS.json hbm_gbs)")
    out["batch"] = b_out.value
    out["other_kernel"] = other
    if gem:
        # split precision: 3 BF16/TF32 MMA passes over the real embedding (4x the complex flops)
        gem_tfs = sum(fl[i] for i in gem) / (t_gem / 1e3) / 1e12 if t_gem > 0 else None
        out["gemm_buckets"] = {"kernel": "k_gemm_pack + k_gemm_tc (k_gemm_tc_fa: B pack only)", "launches": len(gem),
                               "time_share": t_gem / tot,
                               "algorithmic_tflops": gem_tfs}
    out["top_launches"] = [{"kind": ("gemm" if kind[i] >= 100 else "group") if kind[i] else "bucket",
                            "buckets": max(1, kind[i] % 100), "bag": bag[i],
                            "ms": round(ms[i], 4),
                            "gbs": round(by[i] / (ms[i] / 1e3) / 1e9, 1) if ms[i] > 0 else None,
                            "tflops": round(fl[i] / (ms[i] / 1e3) / 1e12, 2) if ms[i] > 0 else None}
                           for i in sorted(range(n), key=lambda i: -ms[i])[:8]]
    return out


def rel_err(a, ref, n):
    """Relative error with the Porter-Thomas floor: |a - ref| / |ref| when
    |ref|^2 >= 2^-n / 10, else |a - ref| / 2^(-n/2)."""
    floor = 2.0 ** (-n / 2)
    den = abs(ref) if abs(ref) ** 2 >= floor ** 2 / 10 else floor
    return abs(a - ref) / den


def oracle_check(circ, bits, plan, gpu_amp, gpu_per, n_check, cpu_budget_s=20.0):
    """FP64 oracle values of slices 0..n_check-1 of the plan (test
    infrastructure, CPU), one call per slice so the first ones also time the
    CPU baseline; returns the amplitude's error (when every slice is checked),
    the largest per-slice error and the baseline sample."""
    from oracle import oracle

    ref = []
    t_sample, n_sample = 0.0, 0
    for s in range(n_check):
        t0 = time.perf_counter()
        ref.append(oracle.contract(circ, bits, order=plan.order(), mu=plan.sliced(), slices=(s, s + 1)))
        dt = time.perf_counter() - t0
        if t_sample < cpu_budget_s:
            t_sample += dt
            n_sample += 1
    n_sl = len(gpu_per)
    slice_err = max(abs(gpu_per[s] - ref[s]) / abs(ref[s]) if ref[s] != 0 else abs(gpu_per[s])
                    for s in range(n_check))
    amp_ref = sum(ref) if n_check == n_sl else None
    return {"amp_ref": amp_ref,
            "amp_err": rel_err(gpu_amp, amp_ref, circ.n_qubits) if amp_ref is not None else None,
            "slice_err_max": slice_err, "n_checked": n_check,
            "cpu_value": n_sample / t_sample, "cpu_slices": n_sample, "cpu_s": t_sample,
            "cores": oracle.num_threads()}


def run_reference(args, cfg_name):
    """The FP64 oracle timed on the host cores: each step contracts one slice."""
    from oracle import oracle
    from paper_2004_10892_gb300 import inputs, tnq

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    rows, cols, cyc, mb, pmin, pmax = CONFIGS[cfg_name]
    circ = inputs.random_grid_circuit(rows, cols, cyc, 0)
    bits = inputs.random_bitstring(circ.n_qubits, 0)
    plan = tnq.Plan(circ, max_bag_log2=mb, min_p=pmin, max_p=pmax, reorder_every=args.reorder_every,
                    order_trials=args.order_trials)
    order, mu = plan.order(), plan.sliced()
    n_sl = plan.info()["n_slices"]
    oracle.build()
    for w in range(args.warmup):
        oracle.contract(circ, bits, order=order, mu=mu, slices=(w % n_sl, w % n_sl + 1))
    t0 = time.perf_counter()
    for k in range(args.steps):
        s = (args.warmup + k) % n_sl
        oracle.contract(circ, bits, order=order, mu=mu, slices=(s, s + 1))
    dt = time.perf_counter() - t0
    v = args.steps / dt
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "slices/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": f"grid {cfg_name} random circuit, seed 0, p={plan.info()['p']}, one slice per step"},
        "cpu_baseline": {"value": v, "unit": "slices/s", "cores": cores, "kind": "oracle",
                         "sample": "one slice of the workload per step (FP64 bucket elimination, OpenMP over entries)"},
        "e2e": {"value": v, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Batched serving workload: 64 seeded circuits on 5x5..7x7 grids at depths
    1+16+1..1+32+1 (uneven sizes), 16 seeded bitstrings each; plans sliced to
    bags <= 2^26 (order recomputed while slicing, split-precision GEMM chains,
    each plan autotuned before timing). One step = one tnq_amplitudes_batch call
    over all 1024 amplitudes (host bitstrings in, FP64 amplitudes out: every
    plan's batches are enqueued on up to four streams with one synchronisation)."""
    import numpy as np
    import torch

    from oracle import oracle
    from paper_2004_10892_gb300 import build as native_build
    from paper_2004_10892_gb300 import inputs, tnq

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        work = inputs.batched_serving_workload(n_circuits=64, bitstrings_per_circuit=16, seed=0)
        oracle.build()
        sample = [(c, b[0]) for c, b in work if c.n_qubits == 25][:args.steps + args.warmup]
        t0 = None
        for k, (c, b) in enumerate(sample):
            if k == args.warmup:
                t0 = time.perf_counter()
            oracle.contract(c, b)
        dt = time.perf_counter() - t0
        n = len(sample) - args.warmup
        v = n / dt
        line = {"impl": "reference", "metric": "amplitudes/s, batched serving workload", "value": v,
                "unit": "amplitudes/s", "n_gpus": args.gpus, "steps": n, "warmup": args.warmup,
                "ms_per_step": 1e3 * dt / n, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "c128", "data": "synthetic",
                "config": {"workload": "batched: the 5x5 circuits of the 64-circuit workload, one amplitude per step"},
                "cpu_baseline": {"value": v, "unit": "amplitudes/s", "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": "5x5 amplitudes of the batched workload (the smallest circuits)"},
                "e2e": {"value": v, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    torch.cuda.set_device(local)
    native_build.build()
    work = inputs.batched_serving_workload(n_circuits=64, bitstrings_per_circuit=16, seed=1000 * rank)
    prec = {"c64": 0, "bf16x3": 1, "tf32x3": 2}[args.precision]
    t_plan = time.perf_counter()
    plans = [tnq.Plan(c, max_bag_log2=26, max_p=30, precision=prec, gemm_min_k_log2=args.gemm_min_k,
                      reorder_every=args.reorder_every, fuse_min_rank=args.fuse_min_rank) for c, _ in work]
    t_plan = time.perf_counter() - t_plan
    stream = torch.cuda.current_stream()
    free, _ = torch.cuda.mem_get_info()
    ws = torch.empty(int(free * 0.6) // 256 * 256, dtype=torch.uint8, device="cuda")
    t_tune = time.perf_counter()
    tuned = {}
    if args.tune_file and os.path.exists(args.tune_file):
        tuned = json.load(open(args.tune_file))
    if not args.no_autotune:
        for i, ((c, bl), plan) in enumerate(zip(work, plans)):
            key = str(i)
            if key in tuned:
                plan.set_tuning(*tuned[key]["tuning"])
                plan.keep_chains(tuned[key]["kept_chains"])
            else:
                n_sl = plan.info()["n_slices"]
                plan.autotune(bl[0], workspace=ws, max_batch=min(16, n_sl), stream=stream)
                tuned[key] = {"tuning": list(plan.tuning()), "kept_chains": plan.fused_chains()}
        if args.tune_file and rank == 0:
            json.dump(tuned, open(args.tune_file, "w"))
    t_tune = time.perf_counter() - t_tune
    bitlists = [bl for _, bl in work]
    n_amp = sum(len(b) for b in bitlists)
    n_items = sum(len(b) << p.info()["p"] for p, b in zip(plans, bitlists))
    for _ in range(args.warmup):
        amps = tnq.amplitudes_batch(plans, bitlists, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        clk.t0 = t0
        e0.record(stream)
        for _ in range(args.steps):
            amps = tnq.amplitudes_batch(plans, bitlists, workspace=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        clk.t1 = time.perf_counter()
    t_dev = e0.elapsed_time(e1) / 1e3
    t_wall = clk.t1 - t0
    # kernel launches per step: each plan's batches (the largest power-of-two batch whose workspace fits one
    # of the call's four lanes, as tnq_amplitudes_batch picks it) x its launches per batch, + one accumulate each
    region = ws.numel() * 7 // 8 // 4
    launches = 0
    for p, b in zip(plans, bitlists):
        items = len(b) << p.info()["p"]
        B = 1
        while B < items and B < (1 << 16) and p.workspace_bytes(2 * B) <= region:
            B *= 2
        launches += -(-items // B) * (tnq.lib().tnq_internal_launches_per_batch(p.handle, 1, B) + 1)
    launches *= args.steps
    # the plan with the most work: per-launch roofline of one of its batches
    big = max(range(len(plans)), key=lambda i: plans[i].info()["total_flops"])
    roof = None
    if not args.no_profile:
        nb = plans[big].info()["n_slices"]
        roof = launch_roofline(tnq.lib(), plans[big], bitlists[big][0], ws, min(nb, 16), nb, stream, load_peaks(),
                               plans[big].info())
        if roof:
            roof["note"] = f"one batch of the batch's largest plan (circuit {big}, {work[big][0].name})"
    # oracle check of a sample: every 5x5 amplitude of the first 8 circuits of that size
    errs, t_cpu, n_cpu = [], 0.0, 0
    if not args.no_cpu_baseline:
        for i, (c, bl) in enumerate(work):
            if c.n_qubits != 25 or n_cpu >= 8:
                continue
            tt = time.perf_counter()
            ref = oracle.contract(c, bl[0])
            t_cpu += time.perf_counter() - tt
            n_cpu += 1
            errs.append(rel_err(amps[16 * i], ref, c.n_qubits))
    line = {
        "metric": "slice-contractions/s & amplitudes/s, batched serving workload (64 circuits x 16 bitstrings)",
        "value": args.steps * n_items / t_dev, "unit": "slices/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"c64": "c64", "bf16x3": "c64+3xbf16", "tf32x3": "c64+3xtf32"}[args.precision], "data": "synthetic",
        "config": {"workload": "batched: 64 seeded circuits, grids 5x5..7x7, depths 1+16+1..1+32+1, 16 bitstrings "
                               "each, bags <= 2^26, one tnq_amplitudes_batch call per step",
                   "amplitudes_per_step": n_amp, "items_per_step": n_items, "plan_s": t_plan, "autotune_s": t_tune,
                   "precision": args.precision, "reorder_every": args.reorder_every,
                   "l2": "inputs larger than L2 (the large plans stream GBs per batch)"},
        "amplitudes_per_s": args.steps * n_amp / t_dev,
        "time_per_amplitude_s": t_dev / (args.steps * n_amp),
        "rel_err_vs_fp64": max(errs) if errs else None,
        "rel_err_vs_fp64_detail": {"sample": f"first bitstring of {len(errs)} 5x5 circuits", "max": max(errs)
                                   if errs else None},
        "e2e": {"value": args.steps * n_items / t_wall, "unit": "slices/s",
                "h2d_bytes_per_step": sum(len(b) * p.n_qubits for p, b in zip(plans, bitlists)),
                "d2h_bytes_per_step": 16 * n_amp},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": {"value": n_cpu / t_cpu, "unit": "amplitudes/s (5x5 circuits only)",
                         "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{n_cpu} 5x5 amplitudes of the workload"} if n_cpu else None,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_learned(args):
    """Learned slicing proposer against tree-trimming on the 8x8 depth 1+32+1
    circuit (seed 0) at bags <= 2^28: the exact cost model of both plans, and
    their measured contraction speed on the GPU. One step = a fixed batch of 32
    slices of the plan (the full amplitudes have thousands of slices; time per
    amplitude = measured time per slice x 2^p, stated as extrapolated)."""
    import numpy as np
    import torch

    from paper_2004_10892_gb300 import build as native_build
    from paper_2004_10892_gb300 import inputs, learned, tnq
    from paper_2004_10892_gb300.train_proposer import plan_pair

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    native_build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    circ = inputs.random_grid_circuit(8, 8, 32, 0)
    bits = inputs.random_bitstring(64, 0)
    w = np.load(learned.TRAINED)
    t_plan = time.perf_counter()
    tt, ln = plan_pair(circ, w, max_bag_log2=28, max_p=60)
    t_plan = time.perf_counter() - t_plan
    stream = torch.cuda.current_stream()
    n = 32
    res = {}
    for name, plan in (("tree_trimming", tt), ("learned", ln)):
        ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            tnq.contract_sliced(plan, bits, 0, n, workspace=ws, max_batch=n, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            tnq.contract_sliced(plan, bits, 0, n, workspace=ws, max_batch=n, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        i = plan.info()
        res[name] = {"p": i["p"], "tau": i["tau"], "max_bag": i["max_bag"], "total_flops": i["total_flops"],
                     "log2_total_flops": float(np.log2(i["total_flops"])), "flops_per_slice": i["flops_per_slice"],
                     "bytes_per_slice": i["bytes_per_slice"], "slices_per_s": args.steps * n / t,
                     "s_per_amplitude_extrapolated": t / (args.steps * n) * i["n_slices"]}
        del ws
    L, T = res["learned"], res["tree_trimming"]
    line = {
        "metric": "slice-contractions/s & time per amplitude, learned proposer vs tree-trimming, 8x8 d1+32+1",
        "value": L["slices_per_s"], "unit": "slices/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * n / L["slices_per_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": "grid 8x8 depth 1+32+1 (seed 0), bags <= 2^28; a step = 32 slices of the learned "
                               "plan", "weights": "paper_2004_10892_gb300/data/proposer_h128.npy", "plan_s": t_plan,
                   "l2": "inputs larger than L2 (each slice streams hundreds of MB)"},
        "time_per_amplitude_s": L["s_per_amplitude_extrapolated"],
        "learned": L, "tree_trimming": T,
        "learned_vs_tree_trimming": {"log2_total_flops": L["log2_total_flops"] - T["log2_total_flops"],
                                     "time_per_amplitude_ratio": L["s_per_amplitude_extrapolated"] /
                                     T["s_per_amplitude_extrapolated"]},
        "e2e": None, "rel_err_vs_fp64": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 60, about 1 s of GPU time; 5 oracle slices for --impl reference)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tnq", choices=["tnq", "reference"])
    ap.add_argument("--config", default="7x7_d1+32+1", choices=sorted(CONFIGS) + ["batched", "learned"],
                    help="workload; 'batched' = 64 circuits (5x5..7x7 grids, depths 1+16+1..1+32+1) x 16 "
                         "bitstrings per step in one tnq_amplitudes_batch call; 'learned' = the 8x8 depth 1+32+1 "
                         "circuit sliced by the learned proposer against tree-trimming (bags <= 2^28)")
    ap.add_argument("--max-batch", type=int, default=256, help="slices contracted at once")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the FP64 oracle (CPU baseline and the amplitude's error)")
    ap.add_argument("--oracle-slices", type=int, default=0,
                    help="slices checked against the FP64 oracle (0: all, which gives the amplitude's error)")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--precision", default="bf16x3", choices=["c64", "bf16x3", "tf32x3"],
                    help="merged GEMM-shaped buckets on tensor cores in split precision")
    ap.add_argument("--reorder-every", type=int, default=1,
                    help="recompute the greedy order after every this many deletions while slicing (0: never)")
    ap.add_argument("--order-trials", type=int, default=32,
                    help="plan from this many greedy orders (seeded random ties) and keep the cheapest")
    ap.add_argument("--fuse-min-rank", type=int, default=12,
                    help="fuse chains whose intermediate results have >= 2^this entries (0: no fusion)")
    ap.add_argument("--gemm-min-k", type=int, default=4,
                    help="split precision: chains summing >= 2^this values run as GEMMs")
    ap.add_argument("--plain", action="store_true",
                    help="plain complex64 per-slice form: one kernel per bucket, no fusion or leaf absorption, "
                         "one slice per launch (a comparison line, not the headline)")
    ap.add_argument("--tune-file", default=None,
                    help="JSON of the autotuner's kept chains: loaded instead of tuning if it exists, else written "
                         "after tuning (lets a profiler run reuse the decisions of a plain run)")
    ap.add_argument("--split-slices", action="store_true",
                    help="under torchrun: every rank contracts its contiguous share of one amplitude's 2^p slices "
                         "and the FP64 partial sums are all-reduced (strong scaling; Eq. 5)")
    ap.add_argument("--tune-batch", type=int, default=0,
                    help="slices per batch while autotuning (0: the timed batch, so the choice is made at the size "
                         "it is used at)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 5 if args.impl == "reference" else 60

    if args.config == "batched":
        if args.steps is None or args.steps == 60:
            args.steps = 3
        run_batched(args)
        return
    if args.config == "learned":
        if args.steps is None or args.steps == 60:
            args.steps = 10
        run_learned(args)
        return
    if args.impl == "reference":
        run_reference(args, args.config)
        return

    import torch
    import torch.distributed as dist

    from paper_2004_10892_gb300 import build as native_build
    from paper_2004_10892_gb300 import inputs, tnq

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    native_build.build()
    rows, cols, cyc, mb, pmin, pmax = CONFIGS[args.config]
    circ = inputs.random_grid_circuit(rows, cols, cyc, 0)
    bits = inputs.random_bitstring(circ.n_qubits, 0 if args.split_slices else rank)
    t_plan = time.perf_counter()
    prec = {"c64": 0, "bf16x3": 1, "tf32x3": 2}[args.precision]
    if args.plain:
        args.precision, prec, args.max_batch, args.no_autotune = "c64", 0, 1, True
        plan = tnq.Plan(circ, max_bag_log2=mb, min_p=pmin, max_p=pmax, fuse_min_rank=0, leaf_absorb=0,
                        reorder_every=args.reorder_every, order_trials=args.order_trials)
    else:
        plan = tnq.Plan(circ, max_bag_log2=mb, min_p=pmin, max_p=pmax, precision=prec,
                        gemm_min_k_log2=args.gemm_min_k, reorder_every=args.reorder_every,
                        fuse_min_rank=args.fuse_min_rank, order_trials=args.order_trials)
    t_plan = time.perf_counter() - t_plan
    n_sl = plan.info()["n_slices"]
    stream = torch.cuda.current_stream()
    L = tnq.lib()
    # autotune (untimed, part of planning): keep each fused chain only where it measures faster
    t_tune = time.perf_counter()
    n_fused = None
    if args.tune_file and os.path.exists(args.tune_file) and not args.no_autotune:
        with open(args.tune_file) as f:
            tf = json.load(f)
        if "tuning" in tf:
            plan.set_tuning(*tf["tuning"])
        plan.keep_chains(tf["kept_chains"])
        n_fused = len(plan.fused_chains())
    elif not args.no_autotune:
        tb = min(args.tune_batch if args.tune_batch > 0 else args.max_batch, n_sl)
        free, _ = torch.cuda.mem_get_info()
        # (the autotuner lowers the batch itself when the unfused layout does not fit)
        tune_ws = torch.empty(int(0.9 * free) // 256 * 256, dtype=torch.uint8, device="cuda")
        n_fused = plan.autotune(bits, workspace=tune_ws, max_batch=tb, stream=stream)
        del tune_ws
        if args.tune_file and rank == 0:
            with open(args.tune_file, "w") as f:
                json.dump({"tuning": list(plan.tuning()), "kept_chains": plan.fused_chains()}, f)
    t_tune = time.perf_counter() - t_tune
    info = plan.info()
    my_b, my_e = 0, n_sl
    if args.split_slices:
        from paper_2004_10892_gb300.shard import sharded_amplitude, slice_range

        my_b, my_e = slice_range(n_sl, rank, world)
    B = min(args.max_batch, max(my_e - my_b, 1))
    free, _ = torch.cuda.mem_get_info()
    while B > 1 and plan.workspace_bytes(B) > 0.8 * free:
        B //= 2
    ws = torch.empty(plan.workspace_bytes(B), dtype=torch.uint8, device="cuda")

    def one_step():
        if args.split_slices:  # this rank's share of the slices, then one FP64 all-reduce (Eq. 5)
            return sharded_amplitude(lambda b, e: tnq.contract_sliced(plan, bits, b, e, workspace=ws, max_batch=B,
                                                                      stream=stream), n_sl)
        return tnq.contract_sliced(plan, bits, workspace=ws, max_batch=B, stream=stream)

    # warm-up (also captures the CUDA graph)
    for _ in range(args.warmup):
        amp = one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        clk.t0 = t0
        e0.record(stream)
        for _ in range(args.steps):
            amp = one_step()
        e1.record(stream)
        torch.cuda.synchronize()
        clk.t1 = time.perf_counter()
        t_wall = clk.t1 - t0
        if world > 1:
            dist.barrier()
    t_dev = e0.elapsed_time(e1) / 1e3
    if world > 1:
        tt = torch.tensor([t_dev, t_wall], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_dev, t_wall = float(tt[0]), float(tt[1])
    total_slices = args.steps * n_sl * (1 if args.split_slices else world)
    value = total_slices / t_dev
    e2e_value = total_slices / t_wall
    n_batches = (my_e - my_b + B - 1) // B
    L.tnq_internal_launches_per_batch.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32]
    launches = args.steps * n_batches * L.tnq_internal_launches_per_batch(plan.handle, 0, B)

    # live per-launch timing of one batch (CUDA events on the launching stream)
    roof = None
    peaks = load_peaks()
    if not args.no_profile and rank == 0:
        roof = launch_roofline(L, plan, bits, ws, B, n_sl, stream, peaks, info)

    cpu = None
    chk = None
    if rank == 0 and not args.no_cpu_baseline:
        # every slice of the timed amplitude in FP64 on the host cores (the
        # parity check of the headline number); the first ~20 s of it also
        # time the CPU baseline
        amp_chk, per = tnq.contract_sliced(plan, bits, 0, n_sl, workspace=ws, max_batch=B, stream=stream,
                                           per_slice=True)
        n_check = n_sl if args.oracle_slices <= 0 else min(args.oracle_slices, n_sl)
        chk = oracle_check(circ, bits, plan, amp_chk, per, n_check)
        chk["same_as_timed"] = amp_chk == amp
        cpu = {"value": chk["cpu_value"], "unit": "slices/s", "cores": chk["cores"], "kind": "oracle",
               "sample": f"slices 0..{chk['cpu_slices'] - 1} of the same amplitude ({chk['cpu_s']:.1f} s; FP64 "
                         f"bucket elimination, OpenMP over output entries)"}

    if rank == 0:
        h2d = 8 + n_batches * (64 + 8 * ((circ.n_qubits + 31) // 32) * (B + 1))
        d2h = n_batches * 16
        line = {
            "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "strong" if args.split_slices else "weak", "vs_baseline": None,
            "dtype": {"c64": "c64", "bf16x3": "c64+3xbf16", "tf32x3": "c64+3xtf32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"grid {args.config} random circuit (seed 0), " +
                       ("one amplitude per step, its slices split across the GPUs" if args.split_slices
                        else "one amplitude per step per GPU"),
                       "n_qubits": circ.n_qubits, "p": info["p"], "n_slices": n_sl, "tau_full": info["tau_full"],
                       "tau": info["tau"], "max_bag": info["max_bag"], "batch": B,
                       "flops_per_slice": info["flops_per_slice"], "bytes_per_slice": info["bytes_per_slice"],
                       "l2": "inputs larger than L2 (each batch streams GBs)", "plan_s": t_plan,
                       "autotune_s": t_tune, "fused_chains": info["n_fused_groups"],
                       "gemm_buckets": info["n_gemm_buckets"], "precision": args.precision,
                       "form": "plain per-slice" if args.plain else "batched, fused, autotuned",
                       "reorder_every": args.reorder_every, "order_trials": args.order_trials,
                       "tuning": {"gemm_min_k_log2": plan.tuning()[0], "tile_low": plan.tuning()[1]}},
            "time_per_amplitude_s": t_dev / args.steps,
            "rel_err_vs_fp64": chk["amp_err"] if chk else None,
            "rel_err_vs_fp64_detail": {
                "amplitude": chk["amp_err"], "max_slice": chk["slice_err_max"],
                "slices_checked": chk["n_checked"], "oracle_amplitude": [chk["amp_ref"].real, chk["amp_ref"].imag]
                if chk["amp_ref"] is not None else None,
                "rule": "|a - a_fp64| / |a_fp64| if |a_fp64|^2 >= 2^-n/10 else / 2^(-n/2); the amplitude is the "
                        "FP64 sum of every slice (Eq. 5), checked from the same batch configuration as the timed "
                        "steps"} if chk else None,
            "amplitude": [amp.real, amp.imag],
            "e2e": {"value": e2e_value, "unit": "slices/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
