"""Benchmark of the spectral-kurtosis flagging path on B300.

Workload (N=1 line): the full-array plain case -- 4 frequencies x N=2048
inputs x M=256 samples x 1525 frames (3.2 GB of 4+4-bit samples, synthetic,
seeded, generated on the device).  One step = one sk_flag call over all 6100
frames (unpack, S1/S2, normalisation, SK~, threshold, mask).  Inputs are 25x
the L2 size, so no flush is needed between steps.

metric: Gsamples/s (1 sample = 1 byte); value = whole-job throughput with
inputs resident in HBM; e2e = the same call on host (pinned) buffers with the
host-to-device upload and the mask/SK download inside the timed region.
After the timed steps a sustained leg streams the same launch back to back for
a few seconds (the regime after the power cap engages: roofline.frac_sustained),
then once more under the configuration tuned for streaming
(tiles_b300_sustained.txt: roofline.frac_sustained_tuned),
and the extras time off-benchmark shapes (`shapes`), the batched mixed
workload, and the serving workload (its full 10 s paced, plus shorter legs).

Under torchrun each rank runs its own 4 frequencies (weak scaling, no
collective in the data path); the timed region is bracketed by barriers and
the max over ranks is taken.

--impl reference times the oracle (plain C/numpy CPU code, test
infrastructure) on a bounded sample of the same workload on the host cores.
"""

from __future__ import annotations

import argparse
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

METRIC = "SK flagging throughput (Gsamples/s, 1 byte/sample)"
UNIT = "Gsamples/s"
N_IN, M_T, N_FREQ, N_FRAMES = 2048, 256, 4, 1525
WORKLOAD = "full_array_plain: {f} freq x N=2048 x M=256 x 1525 frames, 4+4-bit, 3 sigma"
KERNEL_SOURCES = ["paper_1808_10365_b300/csrc/sk_device.cuh",
                  "paper_1808_10365_b300/csrc/sk_path_time.cuh",
                  "paper_1808_10365_b300/csrc/sk_path_input.cuh",
                  "paper_1808_10365_b300/csrc/sk_path_general.cuh",
                  "paper_1808_10365_b300/csrc/sk_api.cu"]
PROFILE_SUMMARY = {0: os.path.join(ROOT, "profiles", "sk_fused_kernel_full_array.json"),
                   1: os.path.join(ROOT, "profiles", "sk_imajor_kernel_full_array.json")}
LAYOUT_SUFFIX = {0: "", 1: ", input-major [frame][input][t]"}
PATH_NAMES = {1: "team", 2: "warp-slice", 3: "row-balanced warp-slice", 4: "general",
              5: "per-input", 6: "stream"}


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6400.0, "fallback"


def profiled_traffic(algorithmic_bytes_per_launch: float, layout: int = 0):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this kernel."""
    try:
        with open(PROFILE_SUMMARY[layout]) as f:
            d = json.load(f)
    except Exception:  # noqa: BLE001
        return None
    if d.get("kernel_hash") != kernel_hash():
        return None
    per_unit = d["dram_bytes_per_launch"] / d["algorithmic_bytes_per_launch"]
    return per_unit * algorithmic_bytes_per_launch


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:  # noqa: BLE001
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:  # noqa: BLE001
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


def physical_index(i: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if i < len(ids) and ids[i].isdigit():
            return int(ids[i])
    return i


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def workload_datasets(rank: int, n_freq: int = N_FREQ, layout: int = 0):
    import dataclasses

    import synth

    # each rank owns its own frequencies (weak scaling): distinct seeds per rank
    ds = synth.full_array_config(n_freq=n_freq, n_frames=N_FRAMES, N=N_IN, M=M_T,
                                 cfg=1 + 1000 * rank)
    return [dataclasses.replace(d, layout=layout) for d in ds] if layout else ds


def static_offset(datasets) -> float:
    import paper_1808_10365_b300 as sk

    sig = np.concatenate([d.sigma for d in datasets])
    return float(np.mean([sk.sk_digitisation_offset(s) for s in sig]))


def cpu_baseline(budget_s: float = 12.0):
    """The oracle as it stands on a bounded sample: 1 frequency x 256 frames of the workload."""
    import oracle
    import synth

    ds = synth.full_array_config(n_freq=1, n_frames=N_FRAMES, N=N_IN, M=M_T)[0]
    nf = 256
    x = ds.generate_cpu(0, nf)
    delta = float(np.mean(oracle.digitisation.delta_of_sigma(ds.sigma)))
    oracle.flag(x[:8], M_T, N_IN, 3.0, delta)  # load the library, first touch
    reps = 0
    t0 = time.perf_counter()
    while True:
        oracle.flag(x, M_T, N_IN, 3.0, delta)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    samples = reps * nf * M_T * N_IN
    cores = oracle.threads()
    # the same path on one core, on a 16-frame sample
    oracle.set_threads(1)
    try:
        n1 = 16
        x1 = x[:n1]
        reps1 = 0
        t1 = time.perf_counter()
        while True:
            oracle.flag(x1, M_T, N_IN, 3.0, delta)
            reps1 += 1
            el1 = time.perf_counter() - t1
            if el1 >= budget_s / 4:
                break
    finally:
        oracle.set_threads(cores)
    return {"value": samples / el / 1e9, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{nf} frames of 1 frequency (N=2048, M=256; {nf * M_T * N_IN / 1e6:.0f} MB) "
                      f"x {reps} repetitions, {el:.1f} s, full oracle path (sums, fp32 and fp64 "
                      f"SK, thresholds, mask)",
            "value_1core": reps1 * n1 * M_T * N_IN / el1 / 1e9,
            "sample_1core": f"{n1} frames x {reps1} repetitions, {el1:.1f} s, 1 thread"}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle

    layout = 1 if args.layout == "input" else 0
    ds = workload_datasets(0, 1, layout)[0]
    # 256 frames (134 MB) a step, the cpu_baseline leg's sample: the oracle's
    # per-call set-up (threshold tables) weighs little against the sums at that size
    nf = 256
    x = ds.generate_cpu(0, nf)
    delta = float(np.mean(oracle.digitisation.delta_of_sigma(ds.sigma)))
    for _ in range(args.warmup):
        oracle.flag(x, M_T, N_IN, 3.0, delta, layout=layout)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.flag(x, M_T, N_IN, 3.0, delta, layout=layout)
    el = time.perf_counter() - t0
    v = args.steps * nf * M_T * N_IN / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": WORKLOAD.format(f=args.freqs) + LAYOUT_SUFFIX[layout],
                       "sample_frames_per_step": nf},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"each step: {nf} frames of 1 frequency of the workload "
                                       f"({nf * M_T * N_IN / 1e6:.0f} MB)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def input_major_bench(n_freq: int, ref_mask, reps: int = 10, dev_index: int = 0):
    """The benchmark workload in the input-major layout [frame][input][t] (the same
    samples, transposed per frame by the generator) through sk_flag; its masks are
    compared with the time-major run's."""
    import torch

    import paper_1808_10365_b300 as sk

    dev = torch.device("cuda", dev_index)
    datasets = workload_datasets(0, n_freq, layout=1)
    F = sum(d.n_frames for d in datasets)
    nbytes = F * M_T * N_IN
    d_in = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    off = 0
    for d in datasets:
        d.generate_gpu(d_in[off:off + d.nbytes])
        off += d.nbytes
    d_sk = torch.empty(F, dtype=torch.float32, device=dev)
    d_mask = torch.empty(F, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N_IN, M_T, 3.0, static_offset(datasets), layout=1,
                             device=dev_index)
    st = torch.cuda.Stream(dev)
    for _ in range(3):
        sk.sk_flag(plan, d_in, F, d_sk, d_mask, st)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for a, b in ev:
        a.record(st)
        sk.sk_flag(plan, d_in, F, d_sk, d_mask, st)
        b.record(st)
    st.synchronize()
    sk.sk_plan_destroy(plan)
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    same = bool(torch.equal(d_mask, ref_mask)) if ref_mask is not None else None
    del d_in
    torch.cuda.empty_cache()
    alg = nbytes + F * 5
    peak, _ = peaks()
    return {"workload": WORKLOAD.format(f=n_freq) + LAYOUT_SUFFIX[1],
            "value": nbytes / (ms * 1e-3) / 1e9, "unit": UNIT, "ms": ms,
            "roofline_frac": alg / (ms * 1e-3) / 1e9 / peak,
            "masks_identical_to_time_major": same}


def variants_bench(d_in, F: int, delta: float, reps: int = 10, dev_index: int = 0):
    """The benchmark workload (already on the device) through two variants of the plain
    launch: per-input estimates with sk_compute_inputs (SK^_i and one-input flags for
    every input, Eq. originalSK, besides SK~ and the mask), and sk_flag on a plan with
    the Pearson type III false-alarm thresholds."""
    import torch

    import paper_1808_10365_b300 as sk

    dev = torch.device("cuda", dev_index)
    st = torch.cuda.Stream(dev)
    peak, _ = peaks()
    nbytes = F * M_T * N_IN

    def timed(fn):
        for _ in range(3):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            a.record(st)
            fn()
            b.record(st)
        st.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    out = {}
    plan = sk.sk_plan_create(N_IN, M_T, 3.0, delta, device=dev_index)
    sk_in = torch.empty((F, N_IN), dtype=torch.float32, device=dev)
    m_in = torch.empty((F, N_IN), dtype=torch.uint8, device=dev)
    d_sk = torch.empty(F, dtype=torch.float32, device=dev)
    d_mask = torch.empty(F, dtype=torch.uint8, device=dev)
    ms = timed(lambda: sk.sk_compute_inputs(plan, d_in, F, sk_in, m_in, d_sk, d_mask, st))
    sk.sk_plan_destroy(plan)
    alg = nbytes + F * N_IN * 5 + F * 5
    out["independent_estimates"] = {
        "call": "sk_compute_inputs (SK^_i float + one-input flag per input, SK~ + mask per frame)",
        "value": nbytes / (ms * 1e-3) / 1e9, "unit": UNIT, "ms": ms,
        "algorithmic_bytes": alg, "roofline_frac": alg / (ms * 1e-3) / 1e9 / peak}
    del sk_in, m_in
    plan = sk.sk_plan_create(N_IN, M_T, 3.0, delta, flags=sk.SK_THRESH_PEARSON3,
                             device=dev_index)
    ms = timed(lambda: sk.sk_flag(plan, d_in, F, d_sk, d_mask, st))
    sk.sk_plan_destroy(plan)
    out["pearson3_thresholds"] = {
        "call": "sk_flag, SK_THRESH_PEARSON3 plan", "value": nbytes / (ms * 1e-3) / 1e9,
        "unit": UNIT, "ms": ms, "roofline_frac": (nbytes + F * 5) / (ms * 1e-3) / 1e9 / peak,
        "flag_rate": float(d_mask.float().mean().item())}
    return out


def batched_bench(reps: int = 10, dev_index: int = 0, n_frames: int = 500):
    """Mixed workload: 64 frequencies of N=2048 and 64 of N=256, M in {128, 256, 1024}
    per frequency from the seed, 500 frames each (n_frames: a smaller case for
    profiling).  One captured graph of persistent launches (sk_batch_run, one launch
    per N class) against one sk_flag launch per frequency, same buffers."""
    import torch

    import paper_1808_10365_b300 as sk
    import synth

    dev = torch.device("cuda", dev_index)
    datasets = synth.mixed_config(n_frames=n_frames)
    total = sum(d.nbytes for d in datasets)
    buf = torch.empty(total + 16 * len(datasets), dtype=torch.uint8, device=dev)
    items, plans, views = [], [], []
    off = 0
    for d in datasets:
        off = (off + 15) // 16 * 16
        v = buf[off:off + d.nbytes]
        d.generate_gpu(v)
        off += d.nbytes
        delta = float(np.mean([sk.sk_digitisation_offset(x) for x in d.sigma]))
        plan = sk.sk_plan_create(d.N, d.M, 3.0, delta, device=dev_index)
        skv = torch.empty(d.n_frames, dtype=torch.float32, device=dev)
        mask = torch.empty(d.n_frames, dtype=torch.uint8, device=dev)
        plans.append(plan)
        views.append((v, skv, mask))
        items.append((plan, v, d.n_frames, skv, mask))
    batch = sk.sk_batch_create(items, dev_index)
    launches = sk.sk_batch_launches(batch)
    st = torch.cuda.Stream(dev)

    def timed(fn):
        for _ in range(3):
            fn()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        st.synchronize()
        return a.elapsed_time(b) / reps

    ms_batch = timed(lambda: sk.sk_batch_run(batch, st))
    mask_b = [m.clone() for _, _, m in views]

    def plain():
        for (plan, v, n, skv, mask) in items:
            sk.sk_flag(plan, v, n, skv, mask, st)

    ms_plain = timed(plain)
    same = all(bool(torch.equal(a, m)) for a, (_, _, m) in zip(mask_b, views))
    sk.sk_batch_destroy(batch)
    for p in plans:
        sk.sk_plan_destroy(p)
    del buf
    torch.cuda.empty_cache()
    ms_list = sorted({d.M for d in datasets})
    return {"workload": "64 freq x N=2048 + 64 freq x N=256, M per freq from {128,256,1024}, "
                        f"{n_frames} frames each, graph-captured persistent launches",
            "bytes": total, "M_values": ms_list,
            "value": total / (ms_batch * 1e-3) / 1e9, "unit": UNIT, "ms": ms_batch,
            "roofline_frac": (total + 5 * sum(d.n_frames for d in datasets))
            / (ms_batch * 1e-3) / 1e9 / peaks()[0],
            "launches_per_run": launches,
            "plain_value": total / (ms_plain * 1e-3) / 1e9, "plain_ms": ms_plain,
            "plain_launches": len(items), "speedup_vs_plain": ms_plain / ms_batch,
            "masks_identical": same}


def served_pools(pool: int = 32):
    """The 32 served streams' pools of pre-generated frames (24 x N=2048 + 8 x N=256,
    M=256, the synthetic noise and RFI model), host numpy arrays."""
    import synth

    out = []
    for k, N in enumerate([2048] * 24 + [256] * 8):
        s = synth.sub_seed(4, k)
        ds = synth.Dataset(n_frames=pool, M=256, N=N, seed=s, rfi=synth.rfi_plan(s, pool))
        out.append(ds.generate_cpu())
    return out


def served_bench(seconds: float = 2.0, paced: bool = True, dev_index: int = 0,
                 pool: int = 32, threads: int = 0, running_mu: bool = False,
                 by_reference: bool = False, pools=None, warmup_s: float = 0.0):
    """32 streams (24 x N=2048, 8 x N=256), M=256 frames arriving every 0.65536 ms per
    stream with exponential jitter (mean T/4), for `seconds` of simulated time, through
    the continuous-batching server with the running power state, driven by the
    library's load generator (sk_server_replay).  Frames cycle through a pool of
    pre-generated frames per stream.  Latency = submit -> result host-visible.
    The plain reference is one synchronous sk_flag_host call per frame.
    threads: submitter threads of the load generator (0: 4 when paced -- enough
    for the 20 GB/s of arrivals, and fewer spinning cores beside the server's
    own threads -- and 8 flat out).  running_mu: the streams also normalise by the
    running power (SK_RUNNING_MU) instead of each frame's own power.  by_reference:
    frames are submitted with sk_stream_submit_ref from page-locked pools (no copy
    into the server's ring) instead of being copied by sk_stream_submit.  pools: the
    streams' frames (numpy arrays, or page-locked tensors for by_reference; generated
    and pinned here when None).  warmup_s: an unmeasured replay of that many seconds
    over the same pools and server before the measured one."""
    import torch

    import paper_1808_10365_b300 as sk
    import synth

    if threads <= 0:
        threads = 4 if paced else 8

    specs = [2048] * 24 + [256] * 8
    M = 256
    T = M * 2.56e-6
    if pools is None:
        pools = served_pools(pool)
        if by_reference:
            pools = [torch.from_numpy(p).pin_memory() for p in pools]
    n_per = int(seconds / T)
    server = sk.sk_server_create(dev_index, 8 << 30)
    flags = sk.SK_RUNNING_MU if running_mu else sk.SK_RUNNING_OFFSET
    sids = [sk.sk_stream_open(server, N, M, ring_frames=32, flags=flags) for N in specs]
    if warmup_s > 0:
        sk.sk_server_replay(server, sids, pools, max(1, int(warmup_s / T)), T, T / 4,
                            paced=paced, threads=threads, by_reference=by_reference)
    r = sk.sk_server_replay(server, sids, pools, n_per, T, T / 4, paced=paced, threads=threads,
                            by_reference=by_reference)
    for sid in sids:
        sk.sk_stream_close(server, sid)
    sk.sk_server_destroy(server)
    out = {"streams": "24 x N=2048 + 8 x N=256, M=256, running power state"
                      + (", running-mu normalisation" if running_mu else "")
                      + (", frames by reference from page-locked memory" if by_reference
                         else ""),
           "paced": paced, "simulated_s": seconds, "frames": r["frames"], "wall_s": r["wall_s"],
           "value": r["bytes"] / r["wall_s"] / 1e9, "unit": UNIT,
           "realtime_input_gbs": sum(specs) * M / T / 1e9,
           "latency_p50_us": r["latency_p50_us"], "latency_p99_us": r["latency_p99_us"],
           "p99_over_p50": r["latency_p99_us"] / max(r["latency_p50_us"], 1e-9),
           "launches": r["launches"], "frames_per_launch": r["frames"] / max(1, r["launches"]),
           "submit_p50_us": r["submit_p50_us"], "busy_retries": r["busy_retries"],
           "load_generator": f"sk_server_replay, {threads} submitter threads"}
    if by_reference and warmup_s > 0:
        out["warmup"] = (f"{warmup_s:g} s unmeasured replay over the same page-locked pools "
                         "(pinned before the first served leg) and server")
    if paced and not running_mu and not by_reference:
        # plain path on the same frames: one synchronous sk_flag_host per frame
        lat = []
        plans = {N: sk.sk_plan_create(N, M, 3.0, 0.0, device=dev_index) for N in set(specs)}
        hm = torch.zeros(1, dtype=torch.uint8).pin_memory()
        hs = torch.zeros(1, dtype=torch.float32).pin_memory()
        pinned = [torch.from_numpy(p[0]).pin_memory() for p in pools]
        for i in range(640):
            j = i % len(specs)
            t1 = time.perf_counter()
            sk.sk_flag_host(plans[specs[j]], pinned[j], 1, hs, hm)
            lat.append((time.perf_counter() - t1) * 1e6)
        for p in plans.values():
            sk.sk_plan_destroy(p)
        lat = np.sort(np.array(lat[32:]))
        out["plain_latency_p50_us"] = float(lat[len(lat) // 2])
        out["plain_latency_p99_us"] = float(lat[int(0.99 * (len(lat) - 1))])
        out["plain_p99_over_p50"] = out["plain_latency_p99_us"] / out["plain_latency_p50_us"]
        out["plain_max_frames_per_s"] = float(1e6 / lat.mean())
        out["realtime_frames_per_s"] = len(specs) / T
    return out


# Shapes off the benchmark's own: ragged N, small arrays and the general path's shapes
# (the stream path), a shape the general path keeps, N = 8 (mod 16), short integrations
# (8-row tile, a partial last turn) and input-major integration lengths at both ends and
# without a fast path (staged blocks).  (label, N, M, layout); each runs on about 3 GB
# of random bytes, the size of the benchmark's own launch.
OFF_SHAPES = [
    ("time-major N=2047 M=256 (ragged N)", 2047, 256, 0),
    ("time-major N=100 M=100 (stream path)", 100, 100, 0),
    ("time-major N=16 M=256 (stream path)", 16, 256, 0),
    ("time-major N=500 M=100 (stream path)", 500, 100, 0),
    ("time-major N=99 M=101 (general path)", 99, 101, 0),
    ("time-major N=2056 M=256 (N = 8 mod 16)", 2056, 256, 0),
    ("time-major N=520 M=256 (N = 8 mod 16)", 520, 256, 0),
    ("time-major N=2048 M=48 (M = 16 mod 32)", 2048, 48, 0),
    ("time-major N=2048 M=100 (M not a multiple of 16)", 2048, 100, 0),
    ("input-major N=2048 M=64", 2048, 64, 1),
    ("input-major N=2048 M=100 (staged blocks)", 2048, 100, 1),
    ("input-major N=2048 M=4096", 2048, 4096, 1),
]


def shapes_bench(reps: int = 10, dev_index: int = 0, target_bytes: int = 3 << 30):
    """sk_flag on each OFF_SHAPES case: about 3 GB of random bytes (24x L2), 3 warm-up
    launches, then `reps` launches each between its own CUDA events on the launching
    stream; throughput and fraction of the measured copy bandwidth per shape."""
    import torch

    import paper_1808_10365_b300 as sk

    dev = torch.device("cuda", dev_index)
    st = torch.cuda.Stream(dev)
    peak, kind = peaks()
    gen = torch.Generator(device=dev)
    gen.manual_seed(1808)
    out = []
    for label, N, M, layout in OFF_SHAPES:
        F = max(1, target_bytes // (M * N))
        nbytes = F * M * N
        d_in = torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device=dev, generator=gen)
        d_sk = torch.empty(F, dtype=torch.float32, device=dev)
        d_mask = torch.empty(F, dtype=torch.uint8, device=dev)
        plan = sk.sk_plan_create(N, M, 3.0, 0.0, layout=layout, device=dev_index)
        try:
            for _ in range(3):
                sk.sk_flag(plan, d_in, F, d_sk, d_mask, st)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(reps)]
            for a, b in ev:
                a.record(st)
                sk.sk_flag(plan, d_in, F, d_sk, d_mask, st)
                b.record(st)
            st.synchronize()
            taken = PATH_NAMES.get(sk.sk_plan_get_config(plan)["last_path"], "?")
        finally:
            sk.sk_plan_destroy(plan)
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        out.append({"shape": label, "path": taken, "N": N, "M": M, "layout": layout, "frames": F,
                    "bytes": nbytes, "ms": ms, "tb_s": nbytes / (ms * 1e-3) / 1e12,
                    "roofline_frac": (nbytes + 5 * F) / (ms * 1e-3) / 1e9 / peak})
        del d_in, d_sk, d_mask
    torch.cuda.empty_cache()
    return {"peak_gbs": peak, "peak_kind": f"{kind} copy bandwidth", "cases": out}


SUSTAINED_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "paper_1808_10365_b300", "tiles_b300_sustained.txt")


def sustained_config(N: int, M: int, layout: int):
    """The launch configuration tuned for continuous streaming (autotune --sustained)
    of (N, M, layout), as sk_plan_set_config keywords, or None without an entry."""
    if not os.path.exists(SUSTAINED_CACHE):
        return None
    with open(SUSTAINED_CACHE) as f:
        for ln in f:
            v = ln.split()
            if ln.startswith("#") or len(v) != 9:
                continue
            if (int(v[0]), int(v[1]), int(v[2])) == (N, M, layout):
                keys = ("rows", "grid_ctas", "path", "team_log2", "prefetch", "batch_path")
                return dict(zip(keys, (int(t) for t in v[3:])))
    return None


def sustained_leg(sk, plan, d_in, F, d_sk, d_mask, stream, alg_bytes, seconds, dev_index,
                  est_launch_s):
    """Back-to-back sk_flag launches of the benchmark workload for about `seconds`, as a
    deployment that streams continuously runs it: the board's power cap engages after
    tens of milliseconds and the SM clock dips.  Each launch between its own events on
    the launching stream; SM clocks sampled during the leg."""
    import torch

    n = max(20, int(seconds / max(est_launch_s, 1e-5)))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(n)]
    torch.cuda.synchronize(d_in.device)
    with ClockSampler(physical_index(dev_index)) as clk:
        t0 = time.perf_counter()
        for a, b in ev:
            a.record(stream)
            sk.sk_flag(plan, d_in, F, d_sk, d_mask, stream)
            b.record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    ms = [a.elapsed_time(b) for a, b in ev]
    mean_ms = statistics.mean(ms)
    peak, _ = peaks()
    q = len(ms) // 4
    quarters = [statistics.median(ms[i * q:(i + 1) * q]) for i in range(4)]
    mhz = clocks.get("sm_mhz")
    return {"seconds": wall, "launches": n, "mean_launch_ms": mean_ms,
            "achieved_gbs": alg_bytes / (mean_ms * 1e-3) / 1e9,
            "frac": alg_bytes / (mean_ms * 1e-3) / 1e9 / peak,
            "launch_ms_quarter_medians": quarters,
            "launch_ms_min_median_max": [min(ms), statistics.median(ms), max(ms)],
            # launch time x median SM clock: flat across runs if the time follows the clock
            "mean_launch_ms_x_median_sm_mhz": mean_ms * mhz if mhz else None,
            "clocks": clocks}


def run_e2e(sk, plan, d_in, d_mask, F, fb, bytes_per_step, e2e_steps, stream, ws):
    """Same metric through sk_flag_host: pinned host input, upload and download timed."""
    import torch

    h_in = torch.empty(F * fb, dtype=torch.uint8).pin_memory()
    h_in.copy_(d_in)
    h_sk = torch.empty(F, dtype=torch.float32).pin_memory()
    h_mask = torch.empty(F, dtype=torch.uint8).pin_memory()
    sk.sk_flag_host(plan, h_in, F, h_sk, h_mask, stream)
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sk.sk_flag_host(plan, h_in, F, h_sk, h_mask, stream)
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    ok = bool((h_mask.numpy() == d_mask.cpu().numpy()).all())
    return {"value": ws * bytes_per_step * e2e_steps / e2e_s / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": bytes_per_step, "d2h_bytes_per_step": F * 5,
            "steps": e2e_steps, "mask_matches_device": ok}


def run_gpu(args):
    import torch

    import paper_1808_10365_b300 as sk

    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    layout = 1 if args.layout == "input" else 0
    datasets = workload_datasets(rank, args.freqs, layout)
    F = sum(d.n_frames for d in datasets)
    fb = M_T * N_IN
    d_in = torch.empty(F * fb, dtype=torch.uint8, device=dev)
    off = 0
    for d in datasets:
        d.generate_gpu(d_in[off:off + d.nbytes])
        off += d.nbytes
    delta = static_offset(datasets)
    d_sk = torch.empty(F, dtype=torch.float32, device=dev)
    d_mask = torch.empty(F, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N_IN, M_T, 3.0, delta, layout=layout, device=dev.index)
    rows, _ = sk.sk_plan_get_tiles(plan)
    stream = torch.cuda.Stream(dev)
    bytes_per_step = F * fb
    alg_bytes = bytes_per_step + F * (4 + 1)

    # ---- device-resident timing ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(physical_index(dev.index)) as clk:
        # the warm-up runs inside the sampled window, right before the timed steps:
        # starting the sampler leaves the GPU idle for about 0.3 s, and the first
        # launches after an idle gap run slower
        for _ in range(max(args.warmup, 3)):
            sk.sk_flag(plan, d_in, F, d_sk, d_mask, stream)
        stream.synchronize()
        barrier(ws)
        torch.cuda.synchronize(dev)
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        t_all0.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            sk.sk_flag(plan, d_in, F, d_sk, d_mask, stream)
            ev[k][1].record(stream)
        t_all1.record(stream)
        stream.synchronize()
    barrier(ws)
    torch.cuda.synchronize(dev)
    clocks = clk.summary()
    total_ms = t_all0.elapsed_time(t_all1)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(total_ms, ws)
    ms_step = total_ms / args.steps
    value = ws * bytes_per_step * args.steps / (total_ms * 1e-3) / 1e9
    mean_launch_s = statistics.mean(launch_ms) * 1e-3
    peak, peak_kind = peaks()
    achieved = alg_bytes / mean_launch_s / 1e9
    traffic = profiled_traffic(alg_bytes, layout)

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    e2e_steps = min(args.e2e_steps, args.steps)
    if e2e_steps > 0:
        e2e = run_e2e(sk, plan, d_in, d_mask, F, fb, bytes_per_step, e2e_steps, stream, ws)
    # the read path the benchmark launch took (sk_launch_config_t.last_path)
    taken = sk.sk_plan_get_config(plan)["last_path"]
    sustained = sustained_tuned = None
    if args.sustained_seconds > 0:
        sustained = sustained_leg(sk, plan, d_in, F, d_sk, d_mask, stream, alg_bytes,
                                  args.sustained_seconds, dev.index, mean_launch_s)
        # the same leg under the configuration tuned for streaming (its entry in the
        # sustained cache, written by autotune --sustained), run after the first
        cfg = sustained_config(N_IN, M_T, layout)
        if cfg is not None:
            plan_s = sk.sk_plan_create(N_IN, M_T, 3.0, delta, layout=layout, device=dev.index)
            try:
                sk.sk_plan_set_config(plan_s, **cfg)
                sustained_tuned = sustained_leg(sk, plan_s, d_in, F, d_sk, d_mask, stream,
                                                alg_bytes, args.sustained_seconds, dev.index,
                                                mean_launch_s)
                sustained_tuned["config"] = dict(
                    cfg, taken=PATH_NAMES.get(sk.sk_plan_get_config(plan_s)["last_path"]),
                    cache=os.path.basename(SUSTAINED_CACHE))
            finally:
                sk.sk_plan_destroy(plan_s)
    sk.sk_plan_destroy(plan)
    line_tail = dict(e2e=e2e)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(f=args.freqs) + LAYOUT_SUFFIX[layout],
                   "frames_per_step": F,
                   "bytes_per_step": bytes_per_step,
                   "l2": f"inputs {bytes_per_step / 1e9:.1f} GB per rank, > L2 (126 MB): no flush",
                   "parallelism": f"frequency sharding x{ws}, no collective",
                   "mean_offset": delta},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "kernel": ((f"sk_fused_kernel<{rows},2,false,2048,0>" if layout == 0
                                 else "sk_imajor_kernel<8,2,true,0,1>")
                                + f", {PATH_NAMES.get(taken, 'unknown')} path"),
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "mean_launch_ms": mean_launch_s * 1e3,
                     "launch_ms_min_median_max": [min(launch_ms), statistics.median(launch_ms),
                                                  max(launch_ms)],
                     # medians of the four quarters of the timed launches: after about
                     # 70 ms of back-to-back streaming the launches settle about 6 %
                     # slower (sw_power_cap), which the mean includes
                     "launch_ms_quarter_medians": [
                         statistics.median(launch_ms[q * len(launch_ms) // 4:
                                                     max((q + 1) * len(launch_ms) // 4,
                                                         q * len(launch_ms) // 4 + 1)])
                         for q in range(4)]},
        "e2e": line_tail["e2e"],
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if sustained is not None:
        line["roofline"]["frac_sustained"] = sustained["frac"]
        line["sustained"] = sustained
    if sustained_tuned is not None:
        line["roofline"]["frac_sustained_tuned"] = sustained_tuned["frac"]
        line["sustained_tuned"] = sustained_tuned
    if ws == 1 and not args.no_extras:
        if layout == 0:
            line.update(variants_bench(d_in, F, delta, dev_index=dev.index))
        del d_in
        torch.cuda.empty_cache()
        if layout == 0:
            line["input_major"] = input_major_bench(args.freqs, d_mask, dev_index=dev.index)
        line["shapes"] = shapes_bench(dev_index=dev.index)
        line["batched"] = batched_bench(dev_index=dev.index)
        # the served streams' pools, generated once; the by-reference leg's page-locked
        # copies pinned before the first served leg and reused, as a server's long-lived
        # receive buffers would be (freshly pinned pools showed multi-millisecond p99
        # episodes in every one of 8 runs, reused ones in a few)
        pools = served_pools()
        pinned = [torch.from_numpy(p).pin_memory() for p in pools]
        line["served"] = served_bench(args.served_seconds, True, dev.index, pools=pools)
        short = min(args.served_seconds, 2.0)
        line["served_replay"] = served_bench(min(short, 1.0), False, dev.index, pools=pools)
        line["served_running_mu"] = served_bench(short, True, dev.index, running_mu=True,
                                                 pools=pools)
        line["served_by_reference"] = served_bench(short, True, dev.index, by_reference=True,
                                                   pools=pinned, warmup_s=0.5)
        del pinned
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_shape(args):
    """--shape N,M[,layout]: sk_flag alone on about --shape-gb GB of random bytes of that
    shape (a case of the off-benchmark table, or any other), `warmup` launches, then
    `steps` launches each between its own CUDA events; one JSON line with the path the
    plan took and the fraction of the measured copy bandwidth."""
    import torch

    import paper_1808_10365_b300 as sk

    parts = [int(v) for v in args.shape.split(",")]
    N, M = parts[0], parts[1]
    layout = parts[2] if len(parts) > 2 else 0
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(dev)
    peak, kind = peaks()
    F = max(1, int(args.shape_gb * (1 << 30)) // (M * N))
    gen = torch.Generator(device=dev)
    gen.manual_seed(1808)
    d_in = torch.randint(0, 256, (F * M * N,), dtype=torch.uint8, device=dev, generator=gen)
    d_sk = torch.empty(F, dtype=torch.float32, device=dev)
    d_mask = torch.empty(F, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N, M, 3.0, 0.0, layout=layout)
    try:
        for _ in range(args.warmup):
            sk.sk_flag(plan, d_in, F, d_sk, d_mask, st)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for a, b in ev:
            a.record(st)
            sk.sk_flag(plan, d_in, F, d_sk, d_mask, st)
            b.record(st)
        st.synchronize()
        taken = PATH_NAMES.get(sk.sk_plan_get_config(plan)["last_path"], "?")
    finally:
        sk.sk_plan_destroy(plan)
    ms = statistics.median(a.elapsed_time(b) for a, b in ev) if ev else float("nan")
    print(json.dumps({"shape": {"N": N, "M": M, "layout": layout, "frames": F},
                      "path": taken, "steps": args.steps, "warmup": args.warmup,
                      "median_launch_ms": ms, "tb_s": F * M * N / (ms * 1e-3) / 1e12,
                      "roofline_frac": (F * M * N + 5 * F) / (ms * 1e-3) / 1e9 / peak,
                      "peak_kind": f"{kind} copy bandwidth"}))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--freqs", type=int, default=N_FREQ, help="frequencies per rank")
    ap.add_argument("--layout", default="time", choices=["time", "input"],
                    help="sample layout of the timed workload: time-major [frame][t][input] "
                         "or input-major [frame][input][t]")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and served measurements")
    ap.add_argument("--served-seconds", type=float, default=10.0,
                    help="simulated seconds of the paced 32-stream served leg (the serving "
                         "workload's full 10 s by default); the other served legs run "
                         "at most 2 s")
    ap.add_argument("--sustained-seconds", type=float, default=3.0,
                    help="seconds of back-to-back launches of the sustained leg (0: skip)")
    ap.add_argument("--shape", default=None,
                    help="N,M[,layout]: time sk_flag alone on that shape and print its line "
                         "(not the benchmark workload)")
    ap.add_argument("--shape-gb", type=float, default=3.0,
                    help="input size of --shape, in GB (random bytes)")
    args = ap.parse_args(argv)
    if args.shape:
        return run_shape(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
