#!/usr/bin/env python3
"""X-engine benchmark: correlator throughput on one or more GB300s.

One step = one block of synthetic channelised voltages through the whole hot
path, via the C ABI: corr_push (4-bit unpack, corner turn, tensor-core
cross-multiply, integration into int64) and corr_dump (visibilities out).

Default workload: the Tianlai cylinder array size -- 192 inputs (96 dual-pol
receivers), 1024 channels, 8192 spectra per block, 4-bit complex samples in
[time][input][channel] order so the corner turn runs on the GPU, common sky
signal plus receiver noise.  Metric: correlator ops/s, 8 integer ops per
complex multiply-accumulate over the N(N+1)/2 baselines incl. autos, plus the
multiple of real time at 250 MSPS (a C-channel spectrum = 2C real samples).

``--impl reference`` times the plain CPU oracle on the host cores instead,
on a bounded sample of the same workload.

Multi-GPU (torchrun, one rank per GPU): channels are independent, so each
rank integrates its own block with no collective on the data path (weak
scaling); timings are reduced with a max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
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

WORKLOADS = {
    "cylinder192": dict(
        desc="cylinder array: 192 inputs x 1024 channels x 8192 spectra/block, 4-bit complex, "
             "[time][input][channel] order (corner turn on GPU), sky+noise model",
        N=192, C=1024, T=8192, layout=1, kind="sky"),
    "cylinder192s": dict(
        desc="cylinder array, 128-channel slice: 192 inputs x 128 channels x 8192 spectra/block, "
             "4-bit complex, [time][input][channel] order, sky+noise model (profiling size)",
        N=192, C=128, T=8192, layout=1, kind="sky"),
    "dish32": dict(
        desc="dish array: 32 inputs x 1024 channels x 4096 spectra/block, 4-bit complex, "
             "[time][channel][input] payload order, sky+noise model",
        N=32, C=1024, T=4096, layout=0, kind="sky"),
    "dish0": dict(
        desc="dish array, plain: 32 inputs x 256 channels x 1024 spectra/block, 4-bit complex, "
             "[time][channel][input] payload order, i.i.d. Gaussian sigma 2.5 (40 distinct blocks "
             "cycled: 335 MB, larger than L2)",
        N=32, C=256, T=1024, layout=0, kind="gauss", alt_blocks=40, batch_instances=40),
    "dish_stream": dict(
        desc="dish array, streaming integration: 32 inputs x 1024 channels, blocks of 4096 spectra, "
             "32 blocks integrated per dump into int64, 4-bit complex, [time][channel][input] "
             "order, sky+noise model (4 distinct 134 MB blocks cycled)",
        N=32, C=1024, T=4096, layout=0, kind="sky", alt_blocks=4, per_dump=32),
    "dish_stream4": dict(
        desc="dish array, streaming integration, small case: 32 inputs x 1024 channels, blocks of "
             "4096 spectra, 4 blocks integrated per dump into int64, 4-bit complex, "
             "[time][channel][input] order, sky+noise model (4 distinct 134 MB blocks)",
        N=32, C=1024, T=4096, layout=0, kind="sky", alt_blocks=4, per_dump=4),
}
# Mixed arrays correlated as one batch (one persistent launch per run, from a
# CUDA graph) against one launch per array: Gaussian samples as the 32-input
# plain case, [time][channel][input] payload order.
BATCH3 = [(32, 256, 1024), (64, 1024, 4096), (192, 4096, 16384)]
WORKLOADS["batch3"] = dict(
    desc="batched mixed arrays: 32 x 256 x 1024, 64 x 1024 x 4096 and 192 x 4096 x 16384 "
         "(inputs x channels x spectra), 4-bit complex, [time][channel][input] order, "
         "i.i.d. Gaussian sigma 2.5, one persistent cross-multiply per run",
    batch=BATCH3, layout=0, kind="gauss")
# Streaming service: integration requests over mixed arrays arriving as a
# Poisson process, admitted by an HBM budget, continuously batched.
WORKLOADS["service4"] = dict(
    desc="streaming service: requests over 32/192/512-input arrays x 2048 channels, 8-bit "
         "complex (sigma 20, clip 127), 2^k spectra with k uniform in 12..18, 4096-spectrum "
         "blocks, Poisson arrivals at 80% of measured capacity, admitted by an HBM budget",
    service=dict(arrays=[32, 192, 512], C=2048, bits=8, layout=0, kmin=12, kmax=18,
                 block=4096, requests=200, load=0.8, budget_gb=170))
# The F-engine front end (PFB + FFT + Eq. 2 + equaliser) of the cylinder
# array on its own, and the whole FX chain per block.
WORKLOADS["fengine192"] = dict(
    desc="F-engine, cylinder array: 192 8-bit ADC inputs, 1024 channels (2048-sample spectra), "
         "4-tap Hamming-sinc PFB, 8192 spectra/block, 4-bit codes out in [c][i][t] order, "
         "Gaussian ADC noise sigma 16 (2 distinct 3.2 GB blocks cycled)",
    fengine=dict(N=192, C=1024, taps=4, T=8192))
WORKLOADS["fengine192s"] = dict(
    desc="F-engine, cylinder array, 512-spectrum slice: 192 8-bit ADC inputs, 1024 channels, "
         "4-tap PFB, 512 spectra/block (202 MB blocks, larger than L2; profiling size)",
    fengine=dict(N=192, C=1024, taps=4, T=512))
WORKLOADS["ingest192"] = dict(
    desc="packet ingest, cylinder array: 6 F-engines x 32 inputs, 32 bands x 32 channels, "
         "8208-byte packets (8 stacked spectra, CRC-32 checked) assembled into 1024-spectrum "
         "[t][c][i] blocks (24576 packets, 202 MB per block) in a 3-segment ring",
    ingest=dict(n_fids=6, n_inputs_pkt=32, n_xids=32, n_chans_pkt=32, T=1024, segments=3),
    N=192, C=1024, T=1024)
WORKLOADS["fx192"] = dict(
    desc="FX chain, cylinder array: 192 8-bit ADC inputs -> F-engine (1024 channels, 4-tap PFB, "
         "equaliser to 4 bits, [c][i][t]) -> X-engine (all baselines, int64) per block of 8192 "
         "spectra, Gaussian ADC noise plus a common delayed sky signal",
    fengine=dict(N=192, C=1024, taps=4, T=8192), fx=True, N=192, C=1024, T=8192)
METRIC = "X-engine correlator Tops/s at 192 inputs (8 int ops per complex MAC, lower triangle incl. autos)"


def xe_metric(n_inputs):
    """The X-engine metric, named for the workload's input count."""
    return METRIC.replace("at 192 inputs", "at %d inputs" % n_inputs)
INGEST_METRIC = ("packet ingest GB/s: 8208-byte F-engine packets checked and assembled into "
                 "X-engine blocks (192 inputs x 1024 channels)")
FX_METRIC = ("FX correlator Tops/s at 192 inputs: 8-bit ADC samples in, int64 visibilities out "
             "(X-engine ops: 8 per complex MAC, lower triangle incl. autos)")
FE_METRIC = ("F-engine throughput: 8-bit ADC samples/s channelised (192 inputs, 1024 channels, "
             "4-tap PFB, 4-bit codes out)")
ADC_RATE = 250e6  # real samples per second per input (Sec. 2)
PAPER_TOPS = 1.2  # xGPU on one GTX 690 core, >= 96 dual-pol stations (Sec. 2.2); context only
REAL_TIME_RATE = 125e6  # spectra x channels per second per input at 250 MSPS real sampling


def ops_per_block(w):
    return 8 * w["N"] * (w["N"] + 1) // 2 * w["C"] * w["T"]


def ops_per_step(w):
    return ops_per_block(w) * w.get("per_dump", 1)


def executed_flops_per_block(w, bits=4):
    """FLOPs (2 per MAC) the tensor cores issue for one block: every 128 x 128
    block of the real Gram's lower triangle once (diagonal blocks in full), or
    one 128 x 128 tile per group of stacked channels."""
    rows = 2 * w["N"] * (bits // 4)
    if rows <= 64:
        rpc = 2
        while rpc < rows:
            rpc <<= 1
        tiles = -(-w["C"] // (128 // rpc))
        macs = tiles * 128 * 128 * w["T"]
    else:
        nrb = -(-rows // 128)
        macs = w["C"] * nrb * (nrb + 1) // 2 * 128 * 128 * w["T"]
    return 2 * macs


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"],
                    bf16_sus=d.get("bf16_tflops_sustained", d["bf16_tflops"]), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


def kernel_traffic(name, launch_units, **shape):
    """DRAM bytes per launch from a committed ncu summary, if the kernel's
    source is unchanged since the capture and the capture's shape (the keys
    it records, e.g. n_inputs and n_time) matches; scaled to this launch's
    units."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = _profile_entry(path, name, shape)
    return None if d is None else d["dram_bytes"] * launch_units / d["units"]


def _profile_entry(path, name, shape):
    """The entry (or, of a list, the first entry) of a kernel in the committed
    ncu summary whose source is unchanged and whose shape matches."""
    try:
        entries = json.load(open(path)).get(name)
        for d in entries if isinstance(entries, list) else [entries]:
            src = open(os.path.join(ROOT, d["source"]), "rb").read()
            if hashlib.sha256(src).hexdigest() != d["source_sha256"]:
                continue
            if any(k in d.get("shape", {}) and d["shape"][k] != v for k, v in shape.items()):
                continue
            return d
    except Exception:
        pass
    return None


def kernel_metric(name, key, **shape):
    """Another figure of a committed ncu summary (e.g. the tensor pipe's active
    percentage), under the same conditions as kernel_traffic: unchanged kernel
    source and matching capture shape; None otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = _profile_entry(path, name, shape)
    return None if d is None else d.get(key)


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=5)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k] == "Active"})
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows),
                "power_w_median": statistics.median(pw) if pw else None}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo")
    return world, rank, local


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_run(w, seconds, seed=0):
    """A bounded sample (channels x spectra) of workload w sized to take about
    `seconds` of oracle time on all host cores; returns the sample block."""
    import oracle
    from paper_1904_07778_gb300 import synth
    cores = os.cpu_count() or 1
    n, T = w["N"], w["T"]
    per_spectrum = n * (n + 1) // 2  # complex MACs per channel per spectrum
    nch = max(1, min(w["C"], cores))
    t_cal = min(T, 128)
    blk = synth.block(w["kind"], seed, n, nch, t_cal, layout=w["layout"])
    t0 = time.perf_counter()
    oracle.correlate(blk, n, nch, t_cal, layout=w["layout"], threads=cores)
    rate = per_spectrum * nch * t_cal / max(time.perf_counter() - t0, 1e-6)  # CMAC/s
    target = rate * seconds
    if target >= per_spectrum * T * nch:
        ts = T
        nch = int(min(w["C"], max(nch, (target // (per_spectrum * T)) // nch * nch)))
    else:
        ts = int(max(16, min(T, target // (per_spectrum * nch))))
    blk = synth.block(w["kind"], seed + 1, n, nch, ts, layout=w["layout"])
    return blk, nch, ts, cores


def time_oracle(blk, w, nch, ts, cores):
    import oracle
    t0 = time.perf_counter()
    oracle.correlate(blk, w["N"], nch, ts, layout=w["layout"], threads=cores)
    return time.perf_counter() - t0


def run_reference(args, w, world, rank):
    if rank != 0:
        return 0
    budget = max(0.05, min(2.0, args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    blk, nch, ts, cores = cpu_oracle_run(w, budget)
    for _ in range(args.warmup):
        time_oracle(blk, w, nch, ts, cores)
    el = [time_oracle(blk, w, nch, ts, cores) for _ in range(args.steps)]
    ops = 8 * w["N"] * (w["N"] + 1) // 2 * nch * ts
    tot = sum(el)
    v = ops * args.steps / tot / 1e12
    sample = "%d of %d channels x %d of %d spectra per step" % (nch, w["C"], ts, w["T"])
    line = {"impl": "reference", "metric": xe_metric(w["N"]), "value": v, "unit": "Tops/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": w["desc"], "sample": sample},
            "cpu_baseline": {"value": v, "unit": "Tops/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "Tops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args, w, world, rank, local):
    import torch
    from paper_1904_07778_gb300 import build, synth
    build.build()
    from paper_1904_07778_gb300.xengine import CORR_ESTATE as xe_estate
    from paper_1904_07778_gb300.xengine import Correlator

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    N, C, T = w["N"], w["C"], w["T"]
    nb = N * (N + 1) // 2
    nalt = w.get("alt_blocks", 2)
    per_dump = w.get("per_dump", 1)
    with torch.cuda.stream(stream):
        # distinct blocks (2 x 1.5 GiB for the default workload, each far larger
        # than the 129 MB L2; more, smaller ones for the small workloads) cycled
        # so that no step reuses cached input
        blocks = [synth.block_device(w["kind"], 1000 * rank + s, N, C, T, w["layout"], dev)
                  for s in range(nalt)]
        vis = torch.empty((C, nb, 2), dtype=torch.int64, device=dev)
        vis2 = torch.empty_like(vis)
    stream.synchronize()
    cor = Correlator(N, C, T, bits=4, layout=w["layout"], stream=stream.cuda_stream)

    # one step = per_dump pushes and one dump of the integration into device
    # memory; the dump is overlapped (corr_dump_async) and step k waits for
    # step k-1's dump, so every dump completes inside the timed region.  By
    # default each integration is bound to its output buffer (corr_bind), so
    # the visibilities are written there directly and the dump copies nothing;
    # --dump-copy integrates in the context's accumulator and copies out.
    # Several blocks per dump go to one corr_push_many: one persistent
    # cross-multiply over all their tasks (per-block pushes with
    # --per-block-push, and where the library needs a corner turn).
    many = per_dump > 1 and not args.per_block_push

    def step(k, many=many):
        out = vis if k % 2 == 0 else vis2
        if not args.dump_copy:
            cor.bind(out)   # free: its last dump (step k-2) was waited for in step k-1
        if many:
            cor.push_many([blocks[(k * per_dump + p) % nalt] for p in range(per_dump)])
        else:
            for p in range(per_dump):
                cor.push(blocks[(k * per_dump + p) % nalt])
        cor.dump_async(out, reset=True)
        if k > 0:
            cor.dump_wait()

    def drain():
        while cor.dump_wait(check=False) != xe_estate:
            pass

    # pipelined corner turn: the turn of block k+1 on `turn_sms` SMs overlaps
    # the cross-multiply of block k on the others; the split is chosen by a
    # short timed sweep unless given
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    pipe, sweep = 0, {}
    if args.pipeline_sms != 0 and w["layout"] != 2:
        cands = [args.pipeline_sms] if args.pipeline_sms > 0 else [0, 16, 20, 24, 28, 32, 36, 40, 44, 48, 52, 56, 64]

        def try_split(cand):
            cor.set_pipeline(cand)
            for k in range(2):
                step(k)
            drain()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(12):
                step(k)
            drain()
            sweep[cand] = 1e3 * (time.perf_counter() - t0) / 12

        for cand in cands:
            try_split(cand)
        if args.pipeline_sms < 0:  # refine around the best split, by 2 SMs and then by 1
            for d_ in (2, 1):
                best = min(sweep, key=sweep.get)
                for cand in (best - d_, best + d_):
                    if best > 0 and 0 < cand < n_sm and cand not in sweep:
                        try_split(cand)
        pipe = min(sweep, key=sweep.get)
        cor.set_pipeline(pipe)

    for k in range(args.warmup):
        step(k)
    drain()
    cor.set_timing(True)
    s0 = cor.stats()
    sampler = ClockSampler(local) if not args.no_clocks else None
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    e0.record(stream)
    # step k returns once dump k-1 is complete, so the host times between
    # consecutive returns are the device's per-step pace
    t_ret = []
    for k in range(args.steps):
        step(k)
        t_ret.append(time.perf_counter())
    drain()             # the last dump is part of the last step
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    clocks = sampler.stop() if sampler else None
    step_dist = None
    if len(t_ret) > 2:
        iv = sorted(1e3 * (b_ - a_) for a_, b_ in zip(t_ret[1:], t_ret[2:]))
        q = lambda f: iv[min(len(iv) - 1, int(f * len(iv)))]
        step_dist = {"p10": q(0.1), "p50": q(0.5), "p90": q(0.9), "n": len(iv),
                     "clock": "host time between consecutive dump completions (steps 2..K)"}
    barrier(world)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world)
    s1 = cor.stats()
    cor.set_timing(False)

    # the same steps with one push (and one cross-multiply launch) per block,
    # for comparison
    per_block = None
    if many:
        nk = max(10, min(50, args.steps))
        for k in range(3):
            step(k, many=False)
        drain()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for k in range(nk):
            step(k, many=False)
        drain()
        g1.record(stream)
        torch.cuda.synchronize()
        pb_ms = max_over_ranks(g0.elapsed_time(g1) / nk, world)
        per_block = {"ms_per_step": pb_ms, "steps": nk,
                     "value": world * ops_per_step(w) / (pb_ms * 1e-3) / 1e12,
                     "note": "one corr_push (one cross-multiply launch) per block"}

    # end to end through the public API with host buffers: pinned input
    # blocks copied in and the visibilities read back every step
    e2e = None
    if not args.no_e2e:
        hb = [torch.empty(blocks[0].numel(), dtype=torch.uint8, pin_memory=True)
              for _ in range(min(nalt, 2))]
        for h, b in zip(hb, blocks):
            h.copy_(b)
        depth = max(1, min(args.e2e_depth, 3))   # at most 4 dumps outstanding
        hv = [torch.empty((C, nb, 2), dtype=torch.int64, pin_memory=True) for _ in range(depth + 1)]

        # `depth` steps of lookahead: step k queues its pushes and an
        # overlapped dump, then waits for step k-depth's visibilities to reach
        # the host, so a host hiccup shorter than depth steps leaves the
        # copy engine busy
        def step_host(k):
            for p in range(per_dump):
                cor.push(hb[(k * per_dump + p) % len(hb)])
            cor.dump_async(hv[k % (depth + 1)], reset=True)
            if k >= depth:
                cor.dump_wait()

        def drain_host(n_steps):
            for _ in range(min(n_steps, depth)):
                cor.dump_wait()

        nw = max(depth + 1, args.warmup // 4)
        for k in range(nw):
            step_host(k)
        drain_host(nw)
        ke = max(3, min(args.steps, args.e2e_steps))
        cor.set_timing(True)
        se0 = cor.stats()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_k = [t0]
        for k in range(ke):
            step_host(k)
            t_k.append(time.perf_counter())
        drain_host(ke)
        e2e_wall = time.perf_counter() - t0
        se1 = cor.stats()
        cor.set_timing(False)
        # host time of each step (queue its pushes, wait for the previous
        # step's visibilities): shows whether a slow run is slow throughout
        e_iv = sorted(1e3 * (b_ - a_) for a_, b_ in zip(t_k, t_k[1:]))
        # the host link alone: one pinned block in and one result out, timed
        # with events (plain copies, for the e2e floor)
        l_in, l_out = [], []
        dv = torch.empty((C, nb, 2), dtype=torch.int64, device="cuda")
        for _ in range(3):
            g0, g1, g2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            g0.record()
            blocks[0].view(-1).copy_(hb[0], non_blocking=True)
            g1.record()
            hv[0].copy_(dv, non_blocking=True)
            g2.record()
            torch.cuda.synchronize()
            l_in.append(g0.elapsed_time(g1))
            l_out.append(g1.elapsed_time(g2))
        link = {"h2d_gbs": hb[0].numel() / (min(l_in) * 1e-3) / 1e9,
                "d2h_gbs": hv[0].numel() * 8 / (min(l_out) * 1e-3) / 1e9}
        del dv
        e2e_ms = max_over_ranks(1e3 * e2e_wall / ke, world)
        e2e = {"value": world * ops_per_step(w) / (e2e_ms * 1e-3) / 1e12, "unit": "Tops/s",
               "h2d_bytes_per_step": blocks[0].numel() * per_dump, "d2h_bytes_per_step": vis.numel() * 8,
               "ms_per_step": e2e_ms, "steps": ke,
               "step_ms": {"min": e_iv[0], "p50": e_iv[len(e_iv) // 2], "max": e_iv[-1]},
               "copy_in_ms_per_step": (se1["copy_in_ms"] - se0["copy_in_ms"]) / ke,
               "pipeline": "step k's dump overlaps the pushes of the next %d step(s) (corr_dump_async)" % depth,
               "link": dict(link, floor_ms_per_step=max(
                   blocks[0].numel() * per_dump / link["h2d_gbs"] / 1e6,
                   vis.numel() * 8 / link["d2h_gbs"] / 1e6))}

    # A block this small is bound by launch latency; the same blocks as
    # independent arrays of one batch (one persistent cross-multiply launch
    # per run, replayed from a CUDA graph) measure the kernel's throughput.
    inst = None
    if w.get("batch_instances"):
        from paper_1904_07778_gb300.xengine import Batch
        ni = w["batch_instances"]
        with torch.cuda.stream(stream):
            bt = Batch([(N, C, T, 4, w["layout"])] * ni, stream=stream.cuda_stream)
            for k in range(ni):
                bt.set_input(k, blocks[k % nalt])
            for _ in range(3):
                bt.run()
            bt.sync()
            nk = max(20, min(200, args.steps))
            h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0.record(stream)
            for _ in range(nk):
                bt.run()
            h1.record(stream)
            bt.sync()
        b_ms = max_over_ranks(h0.elapsed_time(h1) / nk, world)
        b_bytes = ni * (N * C * T + nb * C * 16)
        inst = {"instances": ni, "runs": nk, "ms_per_run": b_ms,
                "value": world * ni * ops_per_block(w) / (b_ms * 1e-3) / 1e12, "unit": "Tops/s",
                "hbm_gbs": b_bytes / (b_ms * 1e-3) / 1e9,
                "hbm_frac": b_bytes / (b_ms * 1e-3) / 1e9 / peaks()["hbm"],
                "bytes_per_run": b_bytes,
                "launches_per_run": bt.info()["launches_per_run"],
                "note": "%d independent arrays of this shape, distinct blocks (%.0f MB, larger than "
                        "L2), one persistent cross-multiply launch per run (corr_batch, CUDA graph); "
                        "bytes = blocks in + int64 visibilities out" % (ni, ni * N * C * T / 1e6)}
        bt.close()

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        blk, nch, ts, cores = cpu_oracle_run(w, args.cpu_seconds)
        dt = time_oracle(blk, w, nch, ts, cores)
        cpu = {"value": 8 * N * (N + 1) // 2 * nch * ts / dt / 1e12, "unit": "Tops/s",
               "cores": cores, "kind": "oracle",
               "sample": "%d of %d channels x %d of %d spectra (%.1f s)" % (nch, C, ts, T, dt)}

    if rank != 0:
        cor.close()
        return 0
    pk = peaks()
    d = {k: s1[k] - s0[k] for k in s1}
    herk_avg = d["herk_ms"] / max(1, d["timed_herk"])
    turn_avg = d["turn_ms"] / max(1, d["timed_turn"])
    # blocks per cross-multiply launch: one at T <= 65536, or a dump's blocks
    # together (corr_push_many)
    bpl = d["blocks"] / max(1, d["herk_launches"])
    herk_ops = ops_per_block(w) * bpl
    # fp8 dense = 2 x bf16 (the nominal ratio).  The kernel runs in launches of
    # about a millisecond, so the burst figure applies; the fraction of the
    # sustained figure is reported beside it.
    fp8 = 2 * pk["bf16"]
    herk = {"kernel": "herk4_kernel", "bound": "tensor", "unit": "TFLOP/s",
            "achieved": herk_ops / (herk_avg * 1e-3) / 1e12, "peak": fp8,
            "avg_launch_ms": herk_avg, "launches": d["timed_herk"], "sms": n_sm - pipe,
            "peak_note": "fp8 dense = 2 x %s bf16 burst (%.1f TF/s)" % (pk["src"], pk["bf16"]),
            "traffic": kernel_traffic("herk4_kernel", C * bpl, n_inputs=N, n_time=T,
                                      multi_block=bpl > 1),
            "tensor_pipe_active_pct": kernel_metric("herk4_kernel", "tensor_pipe_active_pct",
                                                    n_inputs=N, n_time=T, multi_block=bpl > 1)}
    herk["frac"] = herk["achieved"] / herk["peak"]
    herk["frac_of_sustained"] = herk["achieved"] / (2 * pk["bf16_sus"])
    # what the tensor pipe actually executes (diagonal blocks in full): reported
    # beside the algorithmic rate, never in place of it
    exe = executed_flops_per_block(w) * bpl / (herk_avg * 1e-3) / 1e12
    herk["executed_tflops"] = exe
    herk["executed_frac"] = exe / herk["peak"]
    herk["algorithmic_over_executed"] = ops_per_block(w) / executed_flops_per_block(w)
    kernels = [herk]
    if d["timed_turn"] > 0:  # the payload order is read directly when its rows suit TMA
        tb = 2 * N * C * T
        turn = {"kernel": "turn_persist_kernel" if pipe else "turn_kernel", "bound": "hbm",
                "unit": "GB/s", "sms": pipe or n_sm,
                "achieved": tb / (turn_avg * 1e-3) / 1e9, "peak": pk["hbm"], "avg_launch_ms": turn_avg,
                "launches": d["timed_turn"], "peak_note": "%s HBM copy" % pk["src"],
                "traffic": kernel_traffic("turn_persist_kernel" if pipe else "turn_kernel", N * C * T)}
        turn["frac"] = turn["achieved"] / turn["peak"]
        kernels.append(turn)
    # a tensor-bound kernel confined to part of the GPU, also against that
    # part's share of the peak (HBM bandwidth does not divide by SMs)
    herk["frac_of_its_sms"] = herk["frac"] * n_sm / herk["sms"]
    if N <= 32 and d["timed_turn"] == 0:
        # the dish sizes (4 (N + 1) ops per input byte) are bounded by HBM: the
        # cross-multiply reads the payload-order block itself, so its roofline is
        # the block's bytes (plus the int64 visibilities it writes or adds) over
        # its launch time, against the measured copy bandwidth
        herk_bytes = (N * C * T + (2 if per_dump > 1 else 1) * nb * C * 16 / per_dump) * bpl
        herk.update({"bound": "hbm", "unit": "GB/s", "achieved": herk_bytes / (herk_avg * 1e-3) / 1e9,
                     "peak": pk["hbm"], "peak_note": "%s HBM copy" % pk["src"],
                     "tensor_tflops": herk["achieved"], "tensor_frac": herk["frac"],
                     "bytes_per_launch": herk_bytes})
        herk["frac"] = herk["achieved"] / herk["peak"]
    dom = max(kernels, key=lambda k: k["avg_launch_ms"] * k["launches"])
    roof = {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    for k in ("executed_tflops", "executed_frac", "algorithmic_over_executed", "frac_of_its_sms",
              "frac_of_sustained", "tensor_pipe_active_pct", "tensor_tflops", "tensor_frac",
              "bytes_per_launch"):
        if k in dom:
            roof[k] = dom[k]
    roof["kernel"] = dom["kernel"]
    roof["sms"] = dom["sms"]
    if pipe:
        # the overlapped kernels share HBM: the algorithmic bytes of both
        # (turn read + write, cross-multiply read of the turned block) per step
        step_bytes = (2 * N * C * T + N * C * T) * per_dump
        ms_step_ = ms_max / args.steps
        roof["step_hbm"] = {"bytes_per_step": step_bytes,
                            "achieved_gbs": step_bytes / (ms_step_ * 1e-3) / 1e9,
                            "frac": step_bytes / (ms_step_ * 1e-3) / 1e9 / pk["hbm"]}
        roof["note"] = ("the corner turn of block k+1 on %d SMs overlaps the cross-multiply of "
                        "block k on the other %d; frac is against the whole GPU's peak; step_hbm "
                        "counts both kernels' algorithmic HBM bytes over the step; "
                        "--pipeline-sms 0 runs each alone on every SM"
                        % (pipe, n_sm - pipe))
    ms_step = ms_max / args.steps
    value = world * ops_per_step(w) / (ms_step * 1e-3) / 1e12
    # the input block's bytes over the whole step (each block is read from HBM
    # at least once), against the measured copy bandwidth
    in_bytes = N * C * T * per_dump
    roof["input_bytes_over_step"] = {"bytes_per_step": in_bytes,
                                     "gbs": in_bytes / (ms_step * 1e-3) / 1e9,
                                     "frac": in_bytes / (ms_step * 1e-3) / 1e9 / pk["hbm"]}
    line = {
        "metric": xe_metric(N), "value": value, "unit": "Tops/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_TOPS, "dtype": "u8",
        "data": "synthetic (seeded sky+noise model, device-generated)",
        "config": {"workload": w["desc"], "n_inputs": N, "n_chans": C, "n_time": T,
                   "bits": 4, "layout": ["tci", "tic", "cit"][w["layout"]],
                   "l2": "inputs larger than L2 (%d distinct blocks of %.0f MB cycled)" % (
                       nalt, N * C * T / 1e6),
                   "blocks_per_dump": per_dump,
                   "pushes": ("corr_push_many: the dump's %d blocks in one cross-multiply launch"
                              % per_dump if many else "one corr_push per block"),
                   "dump": ("copied out of the context's accumulator" if args.dump_copy else
                            "in place: each integration bound to its device output buffer "
                            "(corr_bind), the dump copies nothing"),
                   "pipeline": {"turn_sms": pipe, "herk_sms": n_sm - pipe,
                                "sweep_ms_per_step": {str(k_): v for k_, v in sweep.items()},
                                "note": "turn of block k+1 overlaps the cross-multiply of block k "
                                        "(corr_set_pipeline); 0 = one stream" if pipe else
                                        "one stream"},
                   "parallelism": "replica per GPU, channels independent" if world > 1 else "1 GPU"},
        "x_real_time": world * C * T * per_dump / REAL_TIME_RATE / (ms_step * 1e-3),
        "step_ms_distribution": step_dist,
        "wall_ms_per_step": 1e3 * wall / args.steps,
        "gpu_launches": (d["herk_launches"] + d["turn_launches"] + d["norm_launches"]),
        "roofline": roof, "kernels": kernels, "blocks_per_launch": bpl,
        "per_block_pushes": per_block, "batch_of_instances": inst,
        "phase_ms_per_step": {"turn": d["turn_ms"] / args.steps, "herk": d["herk_ms"] / args.steps,
                              "dump_copy": d["dump_ms"] / args.steps,
                              "overlapped": bool(pipe)},
        "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
        "vs_baseline_note": "value / 1.2 Tops/s (xGPU, one GTX 690 core, Sec. 2.2): context only",
    }
    print(json.dumps(line), flush=True)
    cor.close()
    return 0


def run_batch(args, w, world, rank, local):
    """Batched mixed arrays: the graph-replayed single launch, the graph with
    the largest array turned in channel ranges beside the cross-multiply, and
    one launch per array."""
    import torch
    from paper_1904_07778_gb300 import build, synth
    build.build()
    from paper_1904_07778_gb300.xengine import Batch, CorrError

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    shapes = [(n, c, t, 4, w["layout"]) for n, c, t in w["batch"]]
    ops = sum(8 * n * (n + 1) // 2 * c * t for n, c, t in w["batch"])
    # the schedules are timed at creation (the kernels' work does not depend
    # on the sample values), then the inputs are filled
    b = Batch(shapes, tune=True)
    for k, (n, c, t) in enumerate(w["batch"]):
        blk = synth.block_device(w["kind"], 30 + k + 1000 * rank, n, c, t, w["layout"], dev)
        b.set_input(k, blk)
        del blk
    b.sync()
    torch.cuda.empty_cache()

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        b.sync()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        b.sync()
        return max_over_ranks(1e3 * (time.perf_counter() - t0) / steps, world)

    sampler = ClockSampler(local) if not args.no_clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ms_single = timed(b.run, args.steps)
    info_single = b.info()
    ms_plain = timed(b.run_plain, args.steps)
    # pipelined graph: a short timed sweep of the split, then the best one
    sweep = {}
    for sms in (32, 36, 38, 40, 42, 44, 48, 52, 56):
        for ch in (4, 8, 16, 32):
            try:
                b.set_pipeline(sms, ch)
            except CorrError:
                continue
            sweep["%d/%d" % (sms, ch)] = timed(b.run, max(10, args.steps // 20))
    ms_pipe, pipe_cfg, info_pipe = None, None, None
    if sweep:
        pipe_cfg = min(sweep, key=sweep.get)
        sms, ch = (int(x) for x in pipe_cfg.split("/"))
        b.set_pipeline(sms, ch)
        ms_pipe = timed(b.run, args.steps)
        info_pipe = b.info()
    clocks = sampler.stop() if sampler else None
    b.close()
    piped = ms_pipe is not None and ms_pipe < ms_single
    ms_graph = ms_pipe if piped else ms_single
    info = info_pipe if piped else info_single
    if rank != 0:
        return 0
    value = world * ops / (ms_graph * 1e-3) / 1e12
    line = {
        "metric": "X-engine correlator Tops/s, batched mixed arrays (sum over arrays)",
        "value": value, "unit": "Tops/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded i.i.d. Gaussian, device-generated)",
        "config": {"workload": w["desc"], "arrays": w["batch"], "bits": 4, "layout": "tci",
                   "l2": "inputs larger than L2 (13 GB per run)"},
        "graph_form": ("pipelined: the largest array turned in channel ranges on %s (turn SMs / "
                       "ranges) beside the cross-multiply" % pipe_cfg) if piped else "single launch",
        "single_launch_graph": {"value": world * ops / (ms_single * 1e-3) / 1e12,
                                "ms_per_step": ms_single, "schedule": info_single},
        "pipelined_graph": None if ms_pipe is None else {
            "value": world * ops / (ms_pipe * 1e-3) / 1e12, "ms_per_step": ms_pipe,
            "turn_sms_ranges": pipe_cfg, "sweep_ms_per_step": sweep},
        "plain_one_launch_per_array": {"value": world * ops / (ms_plain * 1e-3) / 1e12,
                                       "ms_per_step": ms_plain},
        "batched_over_plain": ms_plain / ms_graph,
        "x_real_time": [c * t / REAL_TIME_RATE / (ms_graph * 1e-3) for n, c, t in w["batch"]],
        "schedule": info, "gpu_launches": info["launches_per_run"] * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_service(args, w, world, rank, local):
    """Poisson request stream through the continuous-batching service."""
    import numpy as np
    import torch
    from paper_1904_07778_gb300 import build, synth
    build.build()
    from paper_1904_07778_gb300.xengine import CORR_OK, CORR_REQ_ACTIVE, CORR_REQ_DONE, Service

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = w["service"]
    C, bits, layout, blk_t = cfg["C"], cfg["bits"], cfg["layout"], cfg["block"]
    n_req = args.service_requests or cfg["requests"]
    # sample data, generated once on the device (outside the timing) and
    # reused cyclically: two blocks per array
    data = {n: [synth.block_device("gauss", 40 + 10 * n + s_, n, C, blk_t, layout, dev, bits=bits)
                for s_ in range(2)] for n in cfg["arrays"]}
    outs = {n: torch.empty((C, n * (n + 1) // 2, 2), dtype=torch.int64, device=dev)
            for n in cfg["arrays"]}
    torch.cuda.synchronize()
    svc = Service(int(cfg["budget_gb"] * 2**30))

    def drain(ids):
        """Push and tick until every request in ids is done and fetched."""
        left = dict(ids)  # id -> [n, blocks pushed, n_blocks]
        while left:
            for rid, st_ in list(left.items()):
                n, pushed, nb = st_
                if pushed < nb and svc.state(rid) == CORR_REQ_ACTIVE:
                    if svc.push(rid, data[n][pushed & 1], check=False) == CORR_OK:
                        st_[1] += 1
            svc.tick()
            for rid, st_ in list(left.items()):
                if svc.state(rid) == CORR_REQ_DONE:
                    svc.fetch(rid, outs[st_[0]])
                    del left[rid]

    # capacity: each array alone, 3 blocks (after one warm-up request)
    per_block = {}
    for n in cfg["arrays"]:
        drain({svc.submit(n, C, bits, layout, blk_t, 1): [n, 0, 1]})
        svc.wait()
        t0 = time.perf_counter()
        drain({svc.submit(n, C, bits, layout, blk_t, 3): [n, 0, 3]})
        svc.wait()
        per_block[n] = (time.perf_counter() - t0) / 3
    rng = np.random.default_rng(2024)
    arrays = rng.choice(cfg["arrays"], size=n_req)
    ks = rng.integers(cfg["kmin"], cfg["kmax"] + 1, size=n_req)
    nblocks = [max(1, (1 << int(k)) // blk_t) for k in ks]
    mean_s = float(np.mean([per_block[int(n)] * nb for n, nb in zip(arrays, nblocks)]))
    rate = cfg["load"] / mean_s  # requests per second
    arrive = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    s0 = svc.stats()
    sampler = ClockSampler(local) if not args.no_clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    t0 = time.perf_counter()
    live = {}  # id -> [n, pushed, n_blocks]
    nxt = 0
    while nxt < n_req or live:
        now = time.perf_counter() - t0
        while nxt < n_req and arrive[nxt] <= now:
            n = int(arrays[nxt])
            live[svc.submit(n, C, bits, layout, blk_t, nblocks[nxt])] = [n, 0, nblocks[nxt]]
            nxt += 1
        for rid, st_ in live.items():
            n, pushed, nb = st_
            if pushed < nb and svc.state(rid) == CORR_REQ_ACTIVE:
                if svc.push(rid, data[n][pushed & 1], check=False) == CORR_OK:
                    st_[1] += 1
        launched = svc.tick()
        for rid in [r for r, st_ in live.items() if svc.state(r) == CORR_REQ_DONE]:
            svc.fetch(rid, outs[live[rid][0]])
            del live[rid]
        if not launched and not live and nxt < n_req:
            time.sleep(max(0.0, min(0.01, arrive[nxt] - (time.perf_counter() - t0))))
    svc.wait()
    wall = time.perf_counter() - t0
    clocks = sampler.stop() if sampler else None
    st = svc.stats()
    svc.close()
    if rank != 0:
        return 0
    ops = st["ops"] - s0["ops"]
    chs = st["chan_spectra"] - s0["chan_spectra"]
    # latency percentiles of the Poisson requests only (the calibration ran first)
    alone_tops = {str(n): 8 * n * (n + 1) // 2 * C * blk_t / per_block[n] / 1e12 for n in cfg["arrays"]}
    line = {
        "metric": "X-engine streaming service: sustained x real time and p50/p99 dump latency",
        "value": chs / REAL_TIME_RATE / wall, "unit": "x real time (250 MSPS)",
        "n_gpus": world, "steps": n_req, "warmup": len(cfg["arrays"]) * 2,
        "ms_per_step": 1e3 * wall / n_req, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded Gaussian, device-generated, "
        "two blocks per array reused cyclically)",
        "config": {"workload": w["desc"], "requests": n_req, "budget_gb": cfg["budget_gb"],
                   "arrival_rate_per_s": rate, "mean_request_gpu_s": mean_s},
        "throughput_tops": ops / wall / 1e12,
        "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"], "max": st["max_ms"],
                       "note": "submit to done, all requests incl. 6 calibration ones"},
        "alone_tops_per_array": alone_tops, "ms_per_block_alone": {str(n): 1e3 * v for n, v in per_block.items()},
        "service": {k: st[k] for k in ("submitted", "completed", "ticks", "launches", "blocks",
                                       "peak_in_use", "budget")},
        "gpu_launches": st["launches"] - s0["launches"], "wall_s": wall, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def fe_flops_per_spectrum(C, taps):
    """Algorithmic FLOPs of one input's spectrum: the taps multiply-adds per
    sample of the filter (2 taps M) and half of one complex M-point FFT at
    the usual 5 M log2 M."""
    M = 2 * C
    return 2 * taps * M + 2.5 * M * math.log2(M)


def fp32_peak_tflops(n_sm, sm_mhz):
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOPs per FMA x clock."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


def adc_device(seed, n_inputs, n_samples, dev, sigma=16.0, common=0.0):
    """Gaussian 8-bit ADC streams drawn on the device (optionally a common
    signal delayed by i samples on input i), in 16-input chunks."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    a = torch.empty((n_inputs, n_samples), dtype=torch.int8, device=dev)
    sky = torch.randn(n_samples + n_inputs, generator=g, device=dev) * common if common > 0 else None
    for i in range(0, n_inputs, 16):
        k = min(16, n_inputs - i)
        v = torch.randn((k, n_samples), generator=g, device=dev) * sigma
        if sky is not None:
            for j in range(k):
                v[j] += sky[n_inputs - (i + j):n_inputs - (i + j) + n_samples]
        a[i:i + k] = torch.clamp(torch.round(v), -127, 127).to(torch.int8)
        del v
    return a


def fe_cpu_baseline(cfg, seconds, fx=False):
    """The F-engine oracle (and the X-engine oracle for the FX chain) on a
    bounded sample: one input pair (all inputs for FX) and as many spectra as
    fit in about `seconds`.  numpy: one host core."""
    import numpy as np
    import oracle
    from oracle import fengine as ofe
    from paper_1904_07778_gb300 import synth
    C, taps = cfg["C"], cfg["taps"]
    n = cfg["N"] if fx else 2
    M = 2 * C
    gain = np.full((C, n), 3000, dtype=np.int64)

    def one(ts):
        adc = synth.adc(7, n, (ts + taps - 1) * M)
        t0 = time.perf_counter()
        out = ofe.fengine(adc, C, taps, ts, gain)
        if fx:
            oracle.correlate(np.ascontiguousarray(out["bytes"]).reshape(-1), n, C, ts,
                             layout=oracle.L_TCI, threads=1)
        return time.perf_counter() - t0

    cal = one(4) / 4
    ts = int(max(4, min(cfg["T"], seconds / max(cal, 1e-9))))
    el = one(ts)
    return ts, n, el


def run_fengine(args, w, world, rank, local):
    """The F-engine alone: device-resident ADC blocks in, 4-bit codes out."""
    import numpy as np
    import torch
    from paper_1904_07778_gb300 import build
    build.build()
    from paper_1904_07778_gb300.fengine import FEngine, fe_gains_from_power

    cfg = w["fengine"]
    N, C, taps, T = cfg["N"], cfg["C"], cfg["taps"], cfg["T"]
    M = 2 * C
    S = (T + taps - 1) * M
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)  # torch work, events and both engines on one stream
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = [adc_device(1000 * rank + k, N, S, dev) for k in range(2)]
    out = torch.empty(C * N * T, dtype=torch.uint8, device=dev)
    power = torch.zeros((C, N), dtype=torch.int64, device=dev)
    f = FEngine(N, C, taps, 0, stream=stream.cuda_stream)
    # calibration pass: Eq. 3 gains from the measured power
    f.set_gains(np.ones((C, N), dtype=np.uint32))
    f.channelise(blocks[0], T, power=power)
    f.sync()
    f.set_gains(fe_gains_from_power(power.cpu().numpy(), T, 2.5))
    for k in range(args.warmup):
        f.channelise(blocks[k % 2], T, out=out)
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(local) if not args.no_clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        f.channelise(blocks[k % 2], T, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)

    # end to end: pinned ADC block in, codes out, every step, on three
    # streams (copy in, channelise, copy out) over depth + 1 buffer slots; the
    # host waits for step k-depth's codes, so copies in and out overlap the
    # channelisation and a short host hiccup leaves the copy engines busy
    e2e = None
    if not args.no_e2e:
        depth = max(1, min(args.e2e_depth, 3))
        ns = depth + 1
        h_adc = torch.empty((N, S), dtype=torch.int8, pin_memory=True)
        h_adc.copy_(blocks[0])
        h_out = [torch.empty(C * N * T, dtype=torch.uint8, pin_memory=True) for _ in range(ns)]
        d_in = blocks + [torch.empty_like(blocks[0]) for _ in range(ns - len(blocks))]
        d_out = [out] + [torch.empty_like(out) for _ in range(ns - 1)]
        cin, cout = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(ns)]
        ev_used = [torch.cuda.Event() for _ in range(ns)]
        ev_out = [torch.cuda.Event() for _ in range(ns)]

        # per-step timing events on each stream (start and end of its work)
        tev = []

        def step(k, timed=False):
            s_ = k % ns
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)] if timed else None
            cin.wait_event(ev_used[s_])
            if timed:
                ev[0].record(cin)
            with torch.cuda.stream(cin):
                d_in[s_].copy_(h_adc, non_blocking=True)
            ev_in[s_].record(cin)
            if timed:
                ev[1].record(cin)
            stream.wait_event(ev_in[s_])
            stream.wait_event(ev_out[s_])
            if timed:
                ev[2].record(stream)
            f.channelise(d_in[s_], T, out=d_out[s_])
            ev_used[s_].record(stream)
            if timed:
                ev[3].record(stream)
            cout.wait_event(ev_used[s_])
            if timed:
                ev[4].record(cout)
            with torch.cuda.stream(cout):
                h_out[s_].copy_(d_out[s_], non_blocking=True)
            ev_out[s_].record(cout)
            if timed:
                ev[5].record(cout)
                tev.append(ev)
            if k >= depth:
                ev_out[(k - depth) % ns].synchronize()

        for k in range(ns + 1):
            step(k)
        torch.cuda.synchronize()
        ke = max(3, min(args.steps, args.e2e_steps))
        barrier(world)
        t0 = time.perf_counter()
        for k in range(ke):
            step(k, timed=True)
        ev_out[(ke - 1) % ns].synchronize()
        e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / ke, world)
        torch.cuda.synchronize()
        med = lambda xs: sorted(xs)[len(xs) // 2]
        phases = {"copy_in_ms": med([e[0].elapsed_time(e[1]) for e in tev]),
                  "channelise_ms": med([e[2].elapsed_time(e[3]) for e in tev]),
                  "copy_out_ms": med([e[4].elapsed_time(e[5]) for e in tev]),
                  "pinned": bool(h_adc.is_pinned() and all(h.is_pinned() for h in h_out)),
                  "note": "medians over the timed steps, CUDA events on each stream"}
        # the host link, one block each way alone and both ways at once
        # (events on the copy streams; the floor of a step is the slower)
        lk = {}
        for name, ins, outs in (("h2d", True, False), ("d2h", False, True), ("both", True, True)):
            best = None
            for _ in range(3):
                torch.cuda.synchronize()
                g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                g0.record(stream)
                cin.wait_event(g0)
                cout.wait_event(g0)
                if ins:
                    with torch.cuda.stream(cin):
                        d_in[0].copy_(h_adc, non_blocking=True)
                if outs:
                    with torch.cuda.stream(cout):
                        h_out[0].copy_(d_out[0], non_blocking=True)
                gi, go = torch.cuda.Event(), torch.cuda.Event()
                gi.record(cin)
                go.record(cout)
                stream.wait_event(gi)
                stream.wait_event(go)
                g1.record(stream)
                torch.cuda.synchronize()
                t_ = g0.elapsed_time(g1)
                best = t_ if best is None else min(best, t_)
            lk[name + "_ms"] = best
        e2e = {"value": world * N * T * M / (e2e_ms * 1e-3) / 1e9, "unit": "Gsample/s",
               "h2d_bytes_per_step": N * S, "d2h_bytes_per_step": C * N * T, "ms_per_step": e2e_ms,
               "steps": ke, "pipeline": "copy-in, channelisation and copy-out on three streams, the "
               "host %d step(s) ahead of the oldest copy-out" % depth,
               "link": dict(lk, h2d_gbs=N * S / lk["h2d_ms"] / 1e6, d2h_gbs=C * N * T / lk["d2h_ms"] / 1e6),
               "phases": phases}
        del h_adc, h_out, d_in, d_out
    f.close()
    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        ts, n_in, el = fe_cpu_baseline(cfg, min(args.cpu_seconds, 20.0))
        cpu = {"value": n_in * ts * M / el / 1e9, "unit": "Gsample/s", "cores": 1, "kind": "oracle",
               "sample": "%d of %d inputs x %d of %d spectra (%.1f s, numpy float64, one core)"
                         % (n_in, N, ts, T, el)}
    flops = N * T * fe_flops_per_spectrum(C, taps)
    tflops = flops / (ms * 1e-3) / 1e12
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = fp32_peak_tflops(n_sm, mhz)
    traffic = kernel_traffic("fengine_kernel", N * T, n_chans=C, taps=taps)
    line = {
        "metric": FE_METRIC, "value": world * N * T * M / (ms * 1e-3) / 1e9, "unit": "Gsample/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Gaussian ADC noise, device-generated)",
        "config": {"workload": w["desc"], "n_inputs": N, "n_chans": C, "taps": taps, "n_spectra": T,
                   "output": "4-bit codes, [c][i][t]",
                   "l2": "inputs larger than L2 (2 distinct %.1f GB blocks cycled)" % (N * S / 1e9),
                   "parallelism": "%d GPU" % world},
        "x_real_time": T * M / ADC_RATE / (ms * 1e-3),
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": tflops / peak, "traffic": traffic, "kernel": "fengine_kernel",
                     "peak_note": "FP32: %d SMs x 128 lanes x 2 x %.0f MHz (median SM clock "
                                  "under load)" % (n_sm, mhz),
                     "flops_per_launch": flops,
                     "hbm_gbs": (N * S + C * N * T) / (ms * 1e-3) / 1e9},
        "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ingest(args, w, world, rank, local):
    """Packets -> blocks on the host cores (the paper's net thread), then the
    end-to-end leg: packets -> blocks -> corr_push -> visibilities."""
    import numpy as np
    from paper_1904_07778_gb300 import build, synth
    build.build()
    from paper_1904_07778_gb300.ingest import PacketRing

    cfg = w["ingest"]
    F, I, X, K, T = cfg["n_fids"], cfg["n_inputs_pkt"], cfg["n_xids"], cfg["n_chans_pkt"], cfg["T"]
    N, C = F * I, X * K
    rng = np.random.default_rng(1000 * rank)
    block = rng.integers(0, 256, (T, C, N), dtype=np.uint8)
    threads = max(1, args.ingest_threads)

    def packets_of(k):
        arr = synth.packets_array(block, F, I, X, K, block_index=k)
        # producer j takes the (Fid, Xid) streams j, j + threads, ... (one
        # receive queue per thread); each stream stays in MCNT order
        stream = arr[:, 6].astype(np.int64) * X + arr[:, 7]
        return arr, [np.ascontiguousarray(arr[stream % threads == j]) for j in range(threads)]

    def run(ring, parts, consumer=None):
        import threading
        got = []

        def prod(a):
            k = 0
            while k < len(a):
                k += ring.push_many(a[k:])
                if k < len(a):
                    time.sleep(0.0002)   # the ring is full: the consumer frees a segment

        th = [threading.Thread(target=prod, args=(a,)) for a in parts]
        for t in th:
            t.start()
        while not got:
            r = ring.next(5)
            if r is not None:
                if consumer:
                    consumer(r)
                got.append(r[1]["n_missing"])
                ring.release()
        for t in th:
            t.join()
        return got[0]

    def stream(batches, on_block=None, after_release=None):
        """The producers push the blocks' packets back to back (thread j its
        streams of every block, in block order) while this thread takes each
        closed block and releases it: the ring's steady state.  on_block(r, k)
        runs before block k is released, after_release(k) after."""
        import threading

        def prod_all(j):
            for _, parts_k in batches:
                a_, i_ = parts_k[j], 0
                while i_ < len(a_):
                    i_ += ring.push_many(a_[i_:])
                    if i_ < len(a_):
                        time.sleep(0.0002)   # the ring is full: the consumer frees a segment

        th = [threading.Thread(target=prod_all, args=(j,)) for j in range(threads)]
        t0 = time.perf_counter()
        for t_ in th:
            t_.start()
        missing = []
        while len(missing) < len(batches):
            r = ring.next(5)
            if r is not None:
                if on_block:
                    on_block(r, len(missing))
                missing.append(r[1]["n_missing"])
                ring.release()
                if after_release:
                    after_release(len(missing) - 1)
        el_ = time.perf_counter() - t0
        for t_ in th:
            t_.join()
        return el_, missing

    porder = args.ingest_layout == "packet"
    ring = PacketRing(F, I, X, K, T, n_segments=cfg["segments"], packet_order=porder)
    stream([packets_of(k) for k in range(args.warmup)])
    # every block has its own packets (block index, MCNTs, CRCs), generated
    # before the timed region: at about 400 MB each, at most 12 blocks
    n_timed = min(args.steps, 12)
    batches = [packets_of(k) for k in range(args.warmup, args.warmup + n_timed)]
    arr = batches[-1][0]
    pkt_bytes = arr.nbytes
    el_s, missing = stream(batches)
    assert not any(missing)
    del batches
    st = ring.stats()
    ms = max_over_ranks(1e3 * el_s / n_timed, world)
    # host copy rate of a block-sized buffer by the same number of threads
    # (disjoint slices): the roofline of the producers' payload copies
    import threading
    src = np.ones(T * C * N, dtype=np.uint8)
    dst = np.empty_like(src)
    step_ = -(-src.size // threads)
    tc = []
    for _ in range(3):
        th = [threading.Thread(target=np.copyto, args=(dst[j:j + step_], src[j:j + step_]))
              for j in range(0, src.size, step_)]
        t0 = time.perf_counter()
        for t_ in th:
            t_.start()
        for t_ in th:
            t_.join()
        tc.append(time.perf_counter() - t0)
    copy_gbs = src.nbytes / min(tc) / 1e9
    payload = T * C * N
    e2e = None
    if not args.no_e2e:
        import torch
        from paper_1904_07778_gb300.xengine import CORR_L_TCI, Correlator
        from paper_1904_07778_gb300.xengine import CORR_L_CIT
        torch.cuda.set_device(local)
        vis = torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, pin_memory=True)
        if porder:
            # packet-order block -> device -> pk_turn -> [c][i][t] -> cross-multiply
            cor = Correlator(N, C, T, bits=4, layout=CORR_L_CIT)
            dev = torch.empty(T * C * N, dtype=torch.uint8, device="cuda")
            cit = torch.empty_like(dev)

            def consume(r):
                dev.copy_(torch.from_numpy(r[0].reshape(-1)), non_blocking=True)
                ring.turn(dev, cit)
                cor.push(cit)
                cor.sync()
        else:
            cor = Correlator(N, C, T, bits=4, layout=CORR_L_TCI)

            def consume(r):
                cor.push(r[0])
                cor.sync()
        base = args.warmup + args.steps
        n_e2e = max(3, min(args.steps, args.e2e_steps))
        if porder:
            # streaming: the producers fill blocks k+1, k+2 while the GPU takes
            # block k; a ring segment is released once its copy to the device
            # is done; each block is dumped (overlapped) into pinned memory
            batches = [packets_of(base + k) for k in range(n_e2e)]
            arr = batches[-1][0]
            vis2 = torch.empty_like(vis).pin_memory()
            copied = torch.cuda.Event()

            def on_block(r, k):
                dev.copy_(torch.from_numpy(r[0].reshape(-1)), non_blocking=True)
                copied.record()
                ring.turn(dev, cit)
                cor.push(cit)
                copied.synchronize()      # the segment's bytes are on the device

            def after_release(k):
                cor.dump_async(vis if k % 2 == 0 else vis2, reset=True)
                if k > 0:
                    cor.dump_wait()

            torch.cuda.synchronize()
            el_e, _ = stream(batches, on_block, after_release)
            t1 = time.perf_counter()
            cor.dump_wait()
            e_ms = 1e3 * (el_e + time.perf_counter() - t1) / n_e2e
            del batches
            mode = "streaming over %d blocks: host assembly of the next blocks overlaps the GPU" % n_e2e
        else:
            ee = []
            for k in range(base, base + n_e2e):
                arr, parts = packets_of(k)
                t0 = time.perf_counter()
                run(ring, parts, consumer=consume)
                cor.dump_into(vis, reset=True)
                ee.append(time.perf_counter() - t0)
            e_ms = 1e3 * sum(ee) / len(ee)
            mode = "one block at a time"
        e2e = {"value": arr.nbytes / (e_ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": payload,
               "d2h_bytes_per_step": vis.numel() * 8, "ms_per_step": e_ms, "steps": n_e2e, "mode": mode,
               "path": ("packets -> ring (packet order) -> device -> pk_turn -> corr_push -> corr_dump"
                        if porder else "packets -> ring -> corr_push (pinned block) -> corr_dump")}
        cor.close()
    ring.close()
    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        from oracle import packets as op
        sample = [row.tobytes() for row in arr[:min(len(arr), 3000)]]
        t0 = time.perf_counter()
        op.assemble(sample, F, I, X, K, T)
        dt = time.perf_counter() - t0
        cpu = {"value": len(sample) * arr.shape[1] / dt / 1e9, "unit": "GB/s", "cores": 1,
               "kind": "oracle", "sample": "%d of %d packets of one block (%.1f s, Python)"
                                           % (len(sample), len(arr), dt)}
    gbs = pkt_bytes / (ms * 1e-3) / 1e9
    line = {
        "metric": INGEST_METRIC,
        "value": world * gbs, "unit": "GB/s", "n_gpus": world, "steps": n_timed,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded random 4-bit codes)",
        "config": {"workload": w["desc"], "producer_threads": threads,
                   "timing": "streaming: %d blocks pushed back to back, each taken and released "
                             "as it closes" % n_timed,
                   "block_layout": "packet order (reordered by pk_turn on the GPU)" if porder
                                   else "[t][c][i] assembled on the host",
                   "host_cores": os.cpu_count(), "parallelism": "%d host" % world},
        "packets_per_s": len(arr) / (ms * 1e-3),
        "x_real_time": payload / (ms * 1e-3) / (N * ADC_RATE / 2),
        "gpu_launches": 0,
        "roofline": {"bound": "host", "achieved": gbs, "peak": copy_gbs, "unit": "GB/s",
                     "frac": gbs / copy_gbs, "traffic": None,
                     "peak_note": "host copy of a block-sized buffer by %d threads (measured); "
                                  "each packet is read by the CRC and copied once" % threads},
        "ring": {k: st[k] for k in ("packets", "blocks", "missing", "busy", "bad_crc")},
        "e2e": e2e, "cpu_baseline": cpu, "clocks": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_ingest(args, w, world, rank):
    """The packet oracle's block assembly (plain Python) on a bounded sample of
    each step's packets: GB/s of packets assembled."""
    if rank != 0:
        return 0
    import numpy as np
    from oracle import packets as op
    from paper_1904_07778_gb300 import synth
    cfg = w["ingest"]
    F, I, X, K, T = cfg["n_fids"], cfg["n_inputs_pkt"], cfg["n_xids"], cfg["n_chans_pkt"], cfg["T"]
    block = np.random.default_rng(0).integers(0, 256, (T, X * K, F * I), dtype=np.uint8)
    arr = synth.packets_array(block, F, I, X, K)
    budget = max(0.2, min(3.0, args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    t0 = time.perf_counter()
    op.assemble([row.tobytes() for row in arr[:200]], F, I, X, K, T)
    n = int(max(50, min(len(arr), 200 * budget / max(time.perf_counter() - t0, 1e-6))))
    sample = [row.tobytes() for row in arr[:n]]
    for _ in range(args.warmup):
        op.assemble(sample, F, I, X, K, T)
    el = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        op.assemble(sample, F, I, X, K, T)
        el.append(time.perf_counter() - t0)
    tot = sum(el)
    v = n * arr.shape[1] * args.steps / tot / 1e9
    desc = "%d of %d packets of a block per step (Python, one core)" % (n, len(arr))
    line = {"impl": "reference", "metric": INGEST_METRIC, "value": v, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": w["desc"], "sample": desc},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_fe(args, w, world, rank):
    """The oracle F-engine (and X-engine, for the FX chain) on the host cores,
    a bounded sample per step."""
    if rank != 0:
        return 0
    cfg = w["fengine"]
    fx = "fx" in w
    budget = max(0.2, min(3.0, args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    M = 2 * cfg["C"]
    for _ in range(args.warmup):
        fe_cpu_baseline(cfg, budget, fx)
    runs = [fe_cpu_baseline(cfg, budget, fx) for _ in range(args.steps)]
    ts, n_in = runs[0][0], runs[0][1]
    tot = sum(r[2] for r in runs)
    if fx:
        v, unit, metric = (8 * n_in * (n_in + 1) // 2 * cfg["C"] * ts * args.steps / tot / 1e12,
                           "Tops/s", FX_METRIC)
    else:
        v, unit, metric = n_in * ts * M * args.steps / tot / 1e9, "Gsample/s", FE_METRIC
    sample = "%d of %d inputs x %d of %d spectra per step (numpy float64, one core)" % (
        n_in, cfg["N"], ts, cfg["T"])
    line = {"impl": "reference", "metric": metric, "value": v, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["desc"], "sample": sample},
            "cpu_baseline": {"value": v, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_fx(args, w, world, rank, local):
    """ADC samples in, visibilities out: F-engine then X-engine per block."""
    import numpy as np
    import torch
    from paper_1904_07778_gb300 import build
    build.build()
    from paper_1904_07778_gb300.fengine import FEngine, fe_gains_from_power
    from paper_1904_07778_gb300.xengine import CORR_L_CIT, Correlator

    cfg = w["fengine"]
    N, C, taps, T = cfg["N"], cfg["C"], cfg["taps"], cfg["T"]
    M = 2 * C
    S = (T + taps - 1) * M
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)  # torch work, events and both engines on one stream
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = [adc_device(2000 * rank + k, N, S, dev, sigma=14.0, common=8.0) for k in range(2)]
    codes = torch.empty(C * N * T, dtype=torch.uint8, device=dev)
    nb = N * (N + 1) // 2
    vis = torch.empty((C, nb, 2), dtype=torch.int64, device=dev)
    power = torch.zeros((C, N), dtype=torch.int64, device=dev)
    f = FEngine(N, C, taps, 0, stream=stream.cuda_stream)
    cor = Correlator(N, C, T, bits=4, layout=CORR_L_CIT, stream=stream.cuda_stream)
    f.set_gains(np.ones((C, N), dtype=np.uint32))
    f.channelise(blocks[0], T, power=power)
    f.sync()
    f.set_gains(fe_gains_from_power(power.cpu().numpy(), T, 2.5))

    def step(k, x_only=False, f_only=False):
        if not x_only:
            f.channelise(blocks[k % 2], T, out=codes)
        if not f_only:
            if not args.dump_copy:
                cor.bind(vis)   # integrate in place: the dump copies nothing
            cor.push(codes)
            cor.dump_into(vis, reset=True)

    def timed(**kw):
        for k in range(args.warmup):
            step(k, **kw)
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            step(k, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / args.steps, world)

    sampler = ClockSampler(local) if not args.no_clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ms = timed()
    clocks = sampler.stop() if sampler else None
    ms_f = timed(f_only=True)
    ms_x = timed(x_only=True)

    e2e = None
    if not args.no_e2e:
        h_adc = torch.empty((N, S), dtype=torch.int8, pin_memory=True)
        h_adc.copy_(blocks[0])
        depth = max(1, min(args.e2e_depth, 3))   # at most 4 dumps outstanding
        ns = depth + 1
        hv = [torch.empty((C, nb, 2), dtype=torch.int64, pin_memory=True) for _ in range(ns)]
        d_in = blocks + [torch.empty_like(blocks[0]) for _ in range(ns - len(blocks))]
        cin = torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(ns)]
        ev_used = [torch.cuda.Event() for _ in range(ns)]

        # the host runs `depth` steps ahead of the oldest outstanding dump
        def step_host(k):
            s_ = k % ns
            cin.wait_event(ev_used[s_])
            with torch.cuda.stream(cin):
                d_in[s_].copy_(h_adc, non_blocking=True)
            ev_in[s_].record(cin)
            stream.wait_event(ev_in[s_])
            f.channelise(d_in[s_], T, out=codes)
            ev_used[s_].record(stream)
            cor.push(codes)
            cor.dump_async(hv[s_], reset=True)
            if k >= depth:
                cor.dump_wait()

        def drain_host(n_steps):
            for _ in range(min(n_steps, depth)):
                cor.dump_wait()

        for k in range(ns + 1):
            step_host(k)
        drain_host(ns + 1)
        torch.cuda.synchronize()
        ke = max(3, min(args.steps, args.e2e_steps))
        barrier(world)
        t0 = time.perf_counter()
        for k in range(ke):
            step_host(k)
        drain_host(ke)
        e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / ke, world)
        e2e = {"value": world * ops_per_block(w) / (e2e_ms * 1e-3) / 1e12, "unit": "Tops/s",
               "h2d_bytes_per_step": N * S, "d2h_bytes_per_step": C * nb * 16,
               "ms_per_step": e2e_ms, "steps": ke,
               "pipeline": "ADC copy-in on its own stream, overlapped dumps (corr_dump_async), the "
               "host %d step(s) ahead of the oldest dump" % depth}
        del h_adc, hv, d_in
    f.close()
    cor.close()
    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        ts, n_in, el = fe_cpu_baseline(cfg, min(args.cpu_seconds, 20.0), fx=True)
        cpu = {"value": 8 * n_in * (n_in + 1) // 2 * C * ts / el / 1e12, "unit": "Tops/s", "cores": 1,
               "kind": "oracle", "sample": "%d inputs x %d of %d spectra (%.1f s, F-engine numpy "
               "float64 + X-engine C oracle, one core)" % (n_in, ts, T, el)}
    flops = N * T * fe_flops_per_spectrum(C, taps)
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    fpk = fp32_peak_tflops(n_sm, mhz)
    line = {
        "metric": FX_METRIC, "value": world * ops_per_block(w) / (ms * 1e-3) / 1e12, "unit": "Tops/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+u8",
        "data": "synthetic (seeded Gaussian ADC noise + common delayed signal, device-generated)",
        "config": {"workload": w["desc"], "n_inputs": N, "n_chans": C, "taps": taps, "n_spectra": T,
                   "l2": "inputs larger than L2 (2 distinct %.1f GB ADC blocks cycled)" % (N * S / 1e9),
                   "dump": ("copied out of the context's accumulator" if args.dump_copy else
                            "in place (corr_bind): the dump copies nothing"),
                   "parallelism": "%d GPU" % world},
        "x_real_time": T * M / ADC_RATE / (ms * 1e-3),
        "phase_ms_per_step": {"fengine": ms_f, "xengine_push_dump": ms_x},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "achieved": flops / (ms_f * 1e-3) / 1e12, "peak": fpk,
                     "unit": "TFLOP/s", "frac": flops / (ms_f * 1e-3) / 1e12 / fpk,
                     "traffic": kernel_traffic("fengine_kernel", N * T, n_chans=C, taps=taps),
                     "kernel": "fengine_kernel",
                     "peak_note": "FP32: %d SMs x 128 lanes x 2 x %.0f MHz" % (n_sm, mhz)},
        "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cylinder192")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--e2e-depth", type=int, default=2,
                    help="steps the host runs ahead of the oldest outstanding dump in the e2e leg (1-3)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--pipeline-sms", type=int, default=-1,
                    help="SMs for the pipelined corner turn (0 = off, -1 = pick by a timed sweep)")
    ap.add_argument("--ingest-threads", type=int, default=16,
                    help="producer threads of the packet-ingest workload")
    ap.add_argument("--ingest-layout", choices=["packet", "tci"], default="packet",
                    help="ring blocks in packet order (reordered on the GPU) or [t][c][i]")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dump-copy", action="store_true",
                    help="X-engine workloads: copy each dump out of the context's accumulator "
                         "instead of integrating in place in the output buffer")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--per-block-push", action="store_true",
                    help="one corr_push per block instead of corr_push_many per dump")
    ap.add_argument("--service-requests", type=int, default=0,
                    help="requests of the service workload (default: its configured count)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    w = WORKLOADS[args.workload]
    world, rank, local = dist_setup()
    if args.impl == "reference" and "fengine" in w:
        rc = run_reference_fe(args, w, world, rank)
    elif args.impl == "reference" and "ingest" in w:
        rc = run_reference_ingest(args, w, world, rank)
    elif args.impl == "reference":
        rc = run_reference(args, w, world, rank)
    elif "fx" in w:
        rc = run_fx(args, w, world, rank, local)
    elif "ingest" in w:
        rc = run_ingest(args, w, world, rank, local)
    elif "fengine" in w:
        rc = run_fengine(args, w, world, rank, local)
    elif "batch" in w:
        rc = run_batch(args, w, world, rank, local)
    elif "service" in w:
        rc = run_service(args, w, world, rank, local)
    else:
        rc = run_gpu(args, w, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
