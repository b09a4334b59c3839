#!/usr/bin/env python
"""Benchmark of the NRX forward pass on the 273-PRB, 4-user, 4-Rx slot
(batch of 8 slots, C=64, R=2, N_it=2), through the C ABI.

One step = one nrx_detect_batch over the batch (DMRS LS + interpolation,
StateInit, 2 CGNN iterations, ReadoutLLRs with masking), inputs resident in
HBM; the L2 is flushed (a 256 MB write) before every timed step.  Prints one
JSON line (rank 0).  Under torchrun each rank runs an independent replica on
its own slots (weak scaling, no data-path collective).

--impl reference times the FP64 CPU oracle on the host cores instead (one slot
of the same workload per step).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2409_02912_b300 import synth  # noqa: E402

WORKLOAD = "mu4_4rx_273prb"
METRIC = "NRX REs/s and p99 slot latency on 1 B300, BF16/FP8 vs FP32 at matched BLER"
UNIT = "REs/s"
FP32_CORE_FLOP_PER_CLK_PER_SM = 256  # 128 FP32 lanes x FMA


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["auto", "fp32", "bf16", "fp16", "fp8"], default="auto")
    ap.add_argument("--no-extras", action="store_true", help="skip latency/compare/e2e/cpu legs")
    ap.add_argument("--batch", type=int, default=0, help="slots per step (0 = the workload's batch of 8)")
    ap.add_argument("--oracle-child", type=int, default=0, help=argparse.SUPPRESS)  # internal: see below
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, \
            "fallback"


def nrx_flops_per_re_ue(net: synth.NetConfig) -> dict:
    """Algorithmic FLOPs per RE and user of each kernel kind (2 per MAC)."""
    C, F, R, m = net.channels, net.in_features, net.res_blocks, net.m_max
    return {
        "state_init": 2 * (F * C + 9 * C),
        "message_passing": 2 * (2 * C * C + (2 * C + 2) * C),
        "residual_block": 2 * (2 * 9 * C + 2 * C * C),
        "readout": 2 * (C * C + C * m),
    }


def kernel_bytes_per_launch(w: synth.Workload, n_slots: int, bits, act_bytes: int) -> dict:
    """Algorithmic DRAM bytes per launch of each kernel kind: every tensor it
    must read or write once (activations of act_bytes per element), halo
    re-reads and other redundancy excluded.  The residual block is averaged
    over the R launches of an iteration (R-1 read z and write z; the last
    reads z and the state and writes the state)."""
    net = w.net
    S = 12 * w.num_prb
    n_dmrs = len(w.dmrs_symbols)
    act = n_slots * w.num_users * synth.NUM_SYMBOLS * S * net.channels * act_bytes
    y = n_slots * net.num_rx_ant * synth.NUM_SYMBOLS * S * 8
    llr = sum((synth.NUM_SYMBOLS - n_dmrs) * S * sum(b) * 4 for b in bits)
    R = net.res_blocks
    return {
        "state_init": y + act,
        "message_passing": 2 * act,
        "residual_block": (2 * (R - 1) + 3) * act / R,
        "readout": act * (synth.NUM_SYMBOLS - n_dmrs) / synth.NUM_SYMBOLS + llr,
    }


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_slot_seconds(slots, W64, net):
    from oracle import nrx_oracle as O
    t0 = time.perf_counter()
    for s in slots:
        c = s.cfg
        O.nrx_forward(s.y, s.dmrs, c.num_users, c.dmrs_symbols, c.bits_per_symbol, W64, net.iterations,
                      net.res_blocks)
    return time.perf_counter() - t0


def bench_weights():
    """(FP32 weights, name): the trained network of the workload when its blob
    is present, else the seeded Gaussian initialisation."""
    from paper_2409_02912_b300 import evaluate
    net = synth.WORKLOADS[WORKLOAD].net
    if os.path.exists(evaluate.TRAINED_MU4):
        with open(evaluate.TRAINED_MU4, "rb") as f:
            return synth.unpack_weights(f.read())[1], os.path.basename(evaluate.TRAINED_MU4)
    return synth.make_weights(net), "seeded Gaussian init (PCG64(42))"


def oracle_child(n_slots: int):
    """Internal (--oracle-child N): time the oracle on the first N slots of
    the workload in this process and print the seconds (the parent starts it
    with one-thread BLAS / OpenMP pools)."""
    w = synth.WORKLOADS[WORKLOAD]
    W64 = {k: v.astype(np.float64) for k, v in bench_weights()[0].items()}
    slots = synth.workload_slots(w, n_slots)
    print(oracle_slot_seconds(slots, W64, w.net), flush=True)


def oracle_single_thread_rate(n_slots: int):
    """REs/s of the oracle on the first n_slots slots in a child process whose
    BLAS and OpenMP pools are limited to one thread; None if it fails."""
    import subprocess
    import sys
    one = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                            "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")}
    env = dict(os.environ, **one, CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", str(n_slots)], env=env,
                           capture_output=True, text=True, timeout=900, cwd=ROOT)
        secs = float(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    return n_slots * res_per_slot(synth.WORKLOADS[WORKLOAD]) / secs


def blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(n) if n else 1
    except Exception:
        return os.cpu_count() or 1


def oracle_cpu_baseline(slots, W64, net, sample: str) -> dict:
    """The FP64 oracle timed on the host cores twice over the same slots: in
    a child process with one-thread BLAS / OpenMP pools, and here with the
    default pools (numpy's matmuls are the only multi-threaded part).
    `value` is the all-core rate; `cores` the BLAS threads that run used;
    `nproc` the host's CPU count."""
    w = synth.WORKLOADS[WORKLOAD]
    n_res = len(slots) * res_per_slot(w)
    single = oracle_single_thread_rate(len(slots))
    allc = n_res / oracle_slot_seconds(slots, W64, net)
    return {"value": allc, "unit": UNIT, "cores": blas_threads(), "nproc": os.cpu_count(), "kind": "oracle",
            "single_thread_value": single, "all_core_value": allc, "sample": sample}


def res_per_slot(w: synth.Workload) -> int:
    return synth.NUM_SYMBOLS * 12 * w.num_prb


# ---- multi-rank bookkeeping (one independent replica per GPU, no data-path collective)

def rank_slot_start(rank: int, batch: int) -> int:
    """First slot index of this rank's batch: ranks draw disjoint seeded slots."""
    return rank * batch


def reduce_max_ms(total_ms: float, world: int, device=None) -> float:
    """Max over ranks of the timed region (the job is as slow as its slowest rank)."""
    if world == 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world: int, steps: int, res_per_step: int, max_total_ms: float) -> float:
    """Whole-job REs/s: REs all ranks processed / the slowest rank's time."""
    return world * steps * res_per_step / (max_total_ms * 1e-3)


def run_reference(args, rank, world):
    """FP64 CPU oracle on the host cores, one slot of the workload per step."""
    if rank != 0:
        return
    w = synth.WORKLOADS[WORKLOAD]
    W64 = {k: v.astype(np.float64) for k, v in bench_weights()[0].items()}
    slots = synth.workload_slots(w, w.batch)
    for i in range(args.warmup):
        oracle_slot_seconds([slots[i % len(slots)]], W64, w.net)
    secs = [oracle_slot_seconds([slots[i % len(slots)]], W64, w.net) for i in range(args.steps)]
    total = sum(secs)
    value = args.steps * res_per_slot(w) / total
    cores = blas_threads()
    single = oracle_single_thread_rate(1)  # the same oracle with one-thread pools, on one slot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "slots_per_step": 1, "users": w.num_users,
                                        "num_rx_ant": w.num_rx_ant, "num_prb": w.num_prb,
                                        "net": "C64 R2 N_it2 m_max6"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "nproc": os.cpu_count(), "kind": "oracle",
                         "single_thread_value": single, "all_core_value": value,
                         "sample": f"{args.steps} slots of {WORKLOAD}, one per step, FP64 numpy oracle "
                                   "(single-thread figure: one more slot in a process with one-thread BLAS / OpenMP pools)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# what each mode computes in, beyond its activation type
PRECISION_NOTE = {
    "bf16": "BF16 activations in HBM; BF16 MMAs on the state (split hi + lo weights in message passing, "
            "BF16 weights in the read-out); FP16 cross-user sum g and its weights; FP16 weights, taps and "
            "intermediates inside the residual blocks; FP32 accumulation",
    "fp16": "FP16 activations, weights and depthwise taps; FP32 MMA accumulation",
    "fp8": "E4M3 MMA operands with per-channel weight and per-row activation scales; FP16 activations in HBM",
    "fp32": "FP32 CUDA-core arithmetic",
}


def traffic_for(kernel: str, precision: str):
    """Per-launch DRAM bytes of `kernel` at the 8-slot batch from the committed
    ncu summary, if neither the kernel source nor a header of the CUDA sources
    has changed since the capture (the caller scales it to its batch: the
    traffic grows with the number of tiles)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[f"{kernel}/{precision}"]
    except (OSError, KeyError, ValueError):
        return None
    return rec["bytes_per_launch"] if kernel_source_sha(rec["source"]) == rec["sha256"] else None


def kernel_source_sha(source: str):
    """SHA-256 over a kernel's .cu file and every header of the CUDA sources."""
    csrc = os.path.join(ROOT, "paper_2409_02912_b300", "csrc")
    files = [os.path.join(csrc, source)] + sorted(glob.glob(os.path.join(csrc, "*.cuh")) +
                                                  glob.glob(os.path.join(csrc, "*.h")))
    h = hashlib.sha256()
    try:
        for f in files:
            h.update(open(f, "rb").read())
    except OSError:
        return None
    return h.hexdigest()


def run_ours(args, rank, world, local):
    import torch

    from paper_2409_02912_b300 import nrx

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = synth.WORKLOADS[WORKLOAD]
    net = w.net
    from paper_2409_02912_b300 import evaluate
    W_bench, weights_name = bench_weights()  # the trained network of this workload, else seeded weights
    blob = synth.pack_weights(net, W_bench)
    batch = args.batch or w.batch
    slots = synth.workload_slots(w, batch, start=rank_slot_start(rank, batch))
    n = len(slots)
    S = 12 * w.num_prb
    y = torch.from_numpy(synth.stack_batch(slots)).to(dev)
    dmrs = torch.from_numpy(np.stack([s.dmrs for s in slots])).to(dev)
    bits = [list(s.cfg.bits_per_symbol) for s in slots]
    nv = [s.cfg.noise_var for s in slots]

    precision = args.precision
    if precision == "auto":
        try:
            nrx.Receiver(blob, net.num_rx_ant, w.num_users, w.num_prb, n, "bf16").close()
            precision = "bf16"
        except nrx.NrxError:
            precision = "fp32"
    rx = nrx.Receiver(blob, net.num_rx_ant, w.num_users, w.num_prb, n, precision)
    n_llr = sum(rx.llr_count(nrx.make_cfgs(1, w.num_prb, w.num_users, w.dmrs_symbols, [0], [1.0])[0], b)
                for b in bits)
    llr = torch.empty(n_llr, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        rx.nrx_detect_batch(y, dmrs, w.dmrs_symbols, bits, out=llr, stream=stream)

    def timed(fn, k):
        ts = []
        for _ in range(k):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ts.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ts]

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    launches_per_step = rx.last_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times = timed(step, args.steps)  # the headline: K steps, no per-kernel events
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # the roofline pass: the same K steps again with a CUDA event around every kernel of
    # this library (they keep a kernel's prologue from overlapping the previous kernel's
    # tail, so this pass is slower; it yields each kernel's launch duration)
    rx.nrx_profile(True)
    rx.nrx_profile_read(reset=True)
    ptimes = timed(step, args.steps)
    rx.nrx_profile(False)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = rx.nrx_profile_read(reset=True)
    total_ms = reduce_max_ms(sum(times), world, dev)
    res_step = n * res_per_slot(w)
    value = aggregate_value(world, args.steps, res_step, total_ms)

    extras = {}
    if not args.no_extras and rank == 0:
        # per-slot latency at batch 1 and batch-8 latency percentiles
        y1, d1, b1 = y[:1], dmrs[:1], bits[:1]
        lat1 = timed(lambda: rx.nrx_detect_batch(y1, d1, w.dmrs_symbols, b1, out=llr, stream=stream), 50)
        # the same call captured once in a CUDA graph and replayed
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            rx.nrx_detect_batch(y1, d1, w.dmrs_symbols, b1, out=llr)
        for _ in range(3):
            graph.replay()
        lat1g = timed(graph.replay, 100)
        extras["latency_us"] = {
            "slot_batch1_p50": 1e3 * float(np.percentile(lat1, 50)),
            "slot_batch1_p99": 1e3 * float(np.percentile(lat1, 99)),
            "slot_batch1_graph_p50": 1e3 * float(np.percentile(lat1g, 50)),
            "slot_batch1_graph_p99": 1e3 * float(np.percentile(lat1g, 99)),
            "batch8_p50": 1e3 * float(np.percentile(times, 50)),
            "batch8_p99": 1e3 * float(np.percentile(times, 99)),
        }
        # the other receivers on the same slots
        cmp = {}
        for other in ("fp32", "bf16", "fp16", "fp8"):
            if other == precision:
                continue
            try:
                rx2 = nrx.Receiver(blob, net.num_rx_ant, w.num_users, w.num_prb, n, other)
            except nrx.NrxError:
                continue
            f = lambda: rx2.nrx_detect_batch(y, dmrs, w.dmrs_symbols, bits, out=llr, stream=stream)
            for _ in range(3):
                f()
            ts = timed(f, max(5, args.steps // 2))
            l1 = timed(lambda: rx2.nrx_detect_batch(y1, d1, w.dmrs_symbols, b1, out=llr, stream=stream), 30)
            cmp[f"nrx_{other}"] = {"value": res_step / (1e-3 * statistics.mean(ts)), "unit": UNIT,
                                   "ms_per_step": statistics.mean(ts),
                                   "slot_batch1_p50_us": 1e3 * float(np.percentile(l1, 50)),
                                   "slot_batch1_p99_us": 1e3 * float(np.percentile(l1, 99))}
            rx2.close()
        # Var-IO heads (Sec. III) on the same slots: same active weights, same work
        import dataclasses
        net_v = dataclasses.replace(net, var_io=True)
        rxv = nrx.Receiver(synth.pack_weights(net_v, synth.make_weights(net_v)), net.num_rx_ant, w.num_users,
                           w.num_prb, n, precision)
        f = lambda: rxv.nrx_detect_batch(y, dmrs, w.dmrs_symbols, bits, out=llr, stream=stream)
        for _ in range(3):
            f()
        ts = timed(f, max(5, args.steps // 2))
        cmp[f"nrx_{precision}_var_io"] = {"value": res_step / (1e-3 * statistics.mean(ts)), "unit": UNIT,
                                          "ms_per_step": statistics.mean(ts)}
        rxv.close()
        f = lambda: rx.lmmse_detect_batch(y, dmrs, w.dmrs_symbols, bits, nv, out=llr, stream=stream)
        for _ in range(3):
            f()
        ts = timed(f, max(5, args.steps // 2))
        l1 = timed(lambda: rx.lmmse_detect_batch(y1, d1, w.dmrs_symbols, b1, nv[:1], out=llr, stream=stream), 30)
        cmp["lmmse_fp32"] = {"value": res_step / (1e-3 * statistics.mean(ts)), "unit": UNIT,
                             "ms_per_step": statistics.mean(ts),
                             "slot_batch1_p50_us": 1e3 * float(np.percentile(l1, 50)),
                             "slot_batch1_p99_us": 1e3 * float(np.percentile(l1, 99))}
        extras["compare"] = cmp
        # end to end through the host-buffer entry point
        y_h = torch.from_numpy(synth.stack_batch(slots)).pin_memory()
        d_h = torch.from_numpy(np.stack([s.dmrs for s in slots])).pin_memory()
        l_h = torch.empty(n_llr, dtype=torch.float32).pin_memory()
        for _ in range(3):
            rx.nrx_detect_batch_host(y_h, d_h, w.dmrs_symbols, bits, l_h, stream=stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            rx.nrx_detect_batch_host(y_h, d_h, w.dmrs_symbols, bits, l_h, stream=stream)
        sync_s = (time.perf_counter() - t0) / args.steps
        # pipelined: every step still uploads its grid and pilots and downloads
        # its LLRs (two output buffers in turn), overlapped with the
        # neighbouring steps' compute; timed from the first upload to the
        # last download
        l_h2 = [l_h, torch.empty(n_llr, dtype=torch.float32).pin_memory()]
        for k in range(3):
            rx.nrx_detect_batch_host_async(y_h, d_h, w.dmrs_symbols, bits, l_h2[k & 1])
        rx.nrx_host_drain()
        t0 = time.perf_counter()
        for k in range(args.steps):
            rx.nrx_detect_batch_host_async(y_h, d_h, w.dmrs_symbols, bits, l_h2[k & 1])
        rx.nrx_host_drain()
        e2e_s = (time.perf_counter() - t0) / args.steps
        extras["e2e"] = {"value": res_step / e2e_s, "unit": UNIT,
                         "h2d_bytes_per_step": int(y_h.numel() * 8 + d_h.numel() * 8),
                         "d2h_bytes_per_step": int(n_llr * 4), "mode": "pipelined host calls",
                         "synchronous_value": res_step / sync_s}
        # matched BLER: the trained network on a coded sweep of the 24-PRB two-user workload
        with open(evaluate.TRAINED_MU2, "rb") as f:
            q = evaluate.compare(f.read())
        snr10 = {k: v["snr_at_10pct"] for k, v in q.items() if not k.startswith("_")}
        ref10 = snr10.get("nrx_fp32")
        extras["quality"] = {
            "workload": "mu2_4rx_24prb coded sweep: 2 users x 16-QAM, 4 Rx, (133,171) K=7 code, 1024-bit blocks",
            "weights": os.path.basename(evaluate.TRAINED_MU2),
            "snr_db_at_10pct_bler": snr10,
            "delta_vs_fp32_db": {k: (None if v is None or ref10 is None else v - ref10) for k, v in snr10.items()},
            "bler": {k: v["bler"] for k, v in q.items() if not k.startswith("_")},
            "snr_db_at_10pct_tbler_ldpc": {k: v.get("snr_at_10pct_tbler_ldpc") for k, v in q.items()
                                           if not k.startswith("_")},
            "tbler_ldpc": {k: v.get("tbler_ldpc") for k, v in q.items() if not k.startswith("_")},
            "snrs_db": q["_sweep"]["snrs"], "blocks_per_point": q["_sweep"]["blocks_per_point"],
            "ldpc": q["_sweep"].get("ldpc")}
        if os.path.exists(evaluate.TRAINED_MU4):  # the benchmarked network on its own workload
            q4 = evaluate.compare(blob, precisions=("fp32", "bf16", "fp16"), sw=evaluate.MU4_SWEEP,
                                  early_exit=False)
            s4 = {k: v["snr_at_10pct"] for k, v in q4.items() if not k.startswith("_")}
            extras["quality"]["mu4_4rx_273prb"] = {
                "workload": "8 x 273 PRB slots' geometry: 4 users x QPSK/16-QAM/64-QAM per user, 4 Rx; "
                            "(133,171) code and LDPC transport blocks",
                "weights": weights_name, "snr_db_at_10pct_bler": s4,
                "delta_vs_fp32_db": {k: (None if v is None or s4.get("nrx_fp32") is None else v - s4["nrx_fp32"])
                                     for k, v in s4.items()},
                "bler": {k: v["bler"] for k, v in q4.items() if not k.startswith("_")},
                "snr_db_at_10pct_tbler_ldpc": {k: v.get("snr_at_10pct_tbler_ldpc") for k, v in q4.items()
                                               if not k.startswith("_")},
                "tbler_ldpc": {k: v.get("tbler_ldpc") for k, v in q4.items() if not k.startswith("_")},
                "snrs_db": q4["_sweep"]["snrs"], "blocks_per_point": q4["_sweep"]["blocks_per_point"],
                "ldpc": q4["_sweep"].get("ldpc")}
        with open(evaluate.TRAINED_MU2_VAR_IO, "rb") as f:
            qv = evaluate.compare(f.read(), precisions=("fp32", "bf16"), early_exit=False)
        extras["quality"]["var_io"] = {
            "weights": os.path.basename(evaluate.TRAINED_MU2_VAR_IO),
            "snr_db_at_10pct_bler": {k: v["snr_at_10pct"] for k, v in qv.items() if not k.startswith("_")},
            "bler": {k: v["bler"] for k, v in qv.items() if not k.startswith("_")}}
        # serving loop under the multi-cell load (16 cells, PRB 24/51/106/273, 1-4 users, Poisson
        # arrivals of one slot per 0.5 ms per cell, 0.5 ms deadline) and at a quarter of it
        from paper_2409_02912_b300 import server as nrx_server
        serving = {}
        for name, cells in (("cells16", 16), ("cells4", 4)):
            srv = nrx_server.Server(blob, net.num_rx_ant, (24, 51, 106, 273), max_users=4, max_batch=8,
                                    precision=precision, deadline_us=500.0, hbm_budget_bytes=24 << 30)
            spec = nrx_server.LoadSpec(cells=cells, seconds=2.0)
            serving[name] = nrx_server.run_load(srv, spec)
            srv.close()
        extras["serving"] = serving
        # CPU baseline: the FP64 oracle on one slot of the same workload
        W64 = {k: v.astype(np.float64) for k, v in W_bench.items()}
        extras["cpu_baseline"] = oracle_cpu_baseline(
            slots[:1], W64, net, f"1 slot of {WORKLOAD} (45864 REs), FP64 numpy oracle, single-thread and all-core")

    # roofline of the dominant kernel: bound by its arithmetic intensity
    pk, src = peaks()
    kern = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    k_ms, k_n = prof[kern]
    per_launch_ms = k_ms / max(k_n, 1)
    flops = nrx_flops_per_re_ue(net)[kern] * n * w.num_users * res_per_slot(w)
    nbytes = kernel_bytes_per_launch(w, n, bits, 4 if precision == "fp32" else 2)[kern]
    if precision == "fp32":
        peak = pk["sm_max_mhz"] * 1e6 * 148 * FP32_CORE_FLOP_PER_CLK_PER_SM / 1e12
        bound, unit, achieved = "alu", "TFLOP/s", flops / (per_launch_ms * 1e-3) / 1e12
        peak_desc = "FP32 CUDA-core FMA rate at the measured max SM clock"
    else:
        ridge = pk["bf16_tflops_sustained"] * 1e12 / (pk["hbm_gbs"] * 1e9)
        if flops / nbytes < ridge:
            bound, unit, peak = "hbm", "GB/s", pk["hbm_gbs"]
            achieved = nbytes / (per_launch_ms * 1e-3) / 1e9
            peak_desc = "measured HBM copy bandwidth"
        else:
            bound, unit, peak = "tensor", "TFLOP/s", pk["bf16_tflops_sustained"]
            achieved = flops / (per_launch_ms * 1e-3) / 1e12
            peak_desc = "measured sustained dense BF16 tensor rate (FP16 has the same rate)"
    roofline = {"bound": bound, "kernel": kern, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "peak_source": f"{src}: {peak_desc}",
                "traffic": (lambda t: None if t is None else t * n / 8)(traffic_for(kern, precision)),
                "flop_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
                "intensity_flop_per_byte": flops / nbytes, "launch_ms": per_launch_ms,
                "kernel_share": {k: prof[k][0] / max(sum(v[0] for v in prof.values()), 1e-12) for k in prof
                                 if prof[k][1] > 0},
                "measured_over": "a second timed pass of the same steps with a CUDA event around each kernel "
                                 "(events keep launches from overlapping, so that pass is slower)",
                "profiled_pass_ms_per_step": sum(ptimes) / len(ptimes)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": precision, "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": n, "users": w.num_users, "num_rx_ant": w.num_rx_ant,
                       "num_prb": w.num_prb, "net": "C64 R2 N_it2 m_max6", "l2": "flushed before each step",
                       "parallelism": f"replicas x{world}",
                       "precision": PRECISION_NOTE.get(precision, precision)},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "roofline": roofline,
        }
        line.update(extras)
        if "e2e" not in line:
            line["e2e"] = None
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.oracle_child:
        oracle_child(args.oracle_child)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
