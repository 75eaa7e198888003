"""Autotuner of the fused kernel's launch configuration.

For each (N, M, layout) it times sk_flag over about 3 GB of device-resident
bytes (the size of a streaming launch: the choice between whole frames and
balanced rows depends on the frames per team) under every launch configuration
the shape admits (sk_launch_config_t):
  * time-major: the read path (team, warp-slice with whole frames per team,
    row-balanced warp-slice), rows per register batch (16, 8) and the L2
    prefetch (on, off);
  * input-major: the read path, the threads per frame (the plan's choice and
    one power of two either side) and the L2 prefetch;
and for time-major N = 2048 shapes also the path of the shape's items inside a
batched launch (team class or warp-slice class, sk_batch_create).  The
configurations are timed round-robin over several rounds (each launch between
its own CUDA events; the median per configuration), so that a drift of the
clock under the board's power cap affects all of them alike.  The default
(AUTO) is kept unless another configuration beats it by more than `margin`.
Results never depend on the configuration (exact integer combination), only
speed does; the input bytes are uniform random, since the kernel's cost does not
depend on their values.

With `sustained_s` > 0 (`--sustained SECONDS`) each configuration instead streams
back to back for that long, the regime of a deployment that runs continuously:
the board then sits at its power cap, and a configuration that does the same work
with less energy runs at a higher clock.  The L2 prefetch of the warp-slice paths,
for one, wins in short bursts and loses over seconds (N = 2048, M = 256: 0.917 of
measured copy bandwidth without it at 1912 MHz, 0.900 with it at 1822 MHz).

The winners go to the cache file that sk_plan_create reads (environment
variable SK_AUTOTUNE_CACHE), one line per shape:
    N M layout rows grid path team_log2 prefetch batch_path

    python -m paper_1808_10365_b300.autotune --out tiles.txt 2048:256:0 2048:256:1
    python -m paper_1808_10365_b300.autotune --sustained 3 --out tiles_sustained.txt 2048:256:0
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics

from . import (SK_PATH_AUTO, SK_PATH_ROW_BALANCED, SK_PATH_STREAM, SK_PATH_TEAM, SK_PATH_WARP_SLICE,
               sk_batch_create, sk_batch_destroy, sk_batch_run, sk_flag, sk_plan_create,
               sk_plan_destroy, sk_plan_get_config, sk_plan_set_config)

PATH_NAMES = {0: "auto", 1: "team", 2: "warp-slice", 3: "row-balanced", 4: "general", 6: "stream",
              5: "per-input"}
FIELDS = ("rows", "grid_ctas", "path", "team_log2", "prefetch", "batch_path")


def candidates(N: int, M: int, layout: int, default_team_log2: int):
    """Launch configurations the shape admits, the default (AUTO) first."""
    base = dict(rows=16 if M % 32 == 0 else 8, grid_ctas=0, path=SK_PATH_AUTO, team_log2=0,
                prefetch=0, batch_path=SK_PATH_AUTO)
    out = [dict(base)]
    paths = (SK_PATH_TEAM, SK_PATH_WARP_SLICE, SK_PATH_ROW_BALANCED)
    if layout == 0:
        # warp slices: 32-row turns (16-row tile), or 16-row turns on the 8-row tile
        # where M = 16 mod 32
        ws = N % 8 == 0 and 256 <= N <= 4096 and M % 16 == 0
        for pf in (0, 1):
            if M % 32 == 0:
                for p in paths if ws else (SK_PATH_TEAM,):
                    out.append(dict(base, rows=16, path=p, prefetch=pf))
                out.append(dict(base, rows=8, path=SK_PATH_TEAM, prefetch=pf))
            elif M % 16 == 0:
                for p in paths if ws else (SK_PATH_TEAM,):
                    out.append(dict(base, rows=8, path=p, prefetch=pf))
            # the stream path: any M, N / gcd(N, 16) <= 512; tried below N = 512 (from
            # N = 256 the warp-slice paths read whole rows)
            if N < 512 and N // math.gcd(N, 16) <= 512:
                out.append(dict(base, path=SK_PATH_STREAM, prefetch=pf))
    elif default_team_log2 > 0:
        teams = [t for t in (default_team_log2 - 1, default_team_log2, default_team_log2 + 1)
                 if 5 <= t <= 8]
        for p in paths:
            for t in teams:
                for pf in (0, 1):
                    out.append(dict(base, path=p, team_log2=t, prefetch=pf))
    uniq = []
    for c in out:
        if c not in uniq:
            uniq.append(c)
    return uniq


def _time_round_robin(fns, reps: int, rounds: int):
    """Median launch time (ms) of each callable, timed round-robin, each launch
    between its own events on the current stream."""
    import torch

    times = [[] for _ in fns]
    for f in fns:
        for _ in range(2):
            f()
    torch.cuda.synchronize()
    for _ in range(rounds):
        for k, f in enumerate(fns):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(reps)]
            for a, b in ev:
                a.record()
                f()
                b.record()
            torch.cuda.synchronize()
            times[k].extend(a.elapsed_time(b) for a, b in ev)
    return [statistics.median(t) for t in times]


def _time_sustained(fns, seconds: float, est_ms: float):
    """Mean launch time (ms) of each callable over about `seconds` of back-to-back
    launches (each launch between its own events): one callable after the other, in
    order and then in reverse, the two means averaged, so that the board's warming
    over the sweep falls on all of them alike."""
    import torch

    n = max(20, int(seconds * 1e3 / max(est_ms, 1e-3)))
    sums = [0.0] * len(fns)
    for order in (range(len(fns)), reversed(range(len(fns)))):
        for k in order:
            f = fns[k]
            for _ in range(3):
                f()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(n)]
            for a, b in ev:
                a.record()
                f()
                b.record()
            torch.cuda.synchronize()
            sums[k] += statistics.mean(a.elapsed_time(b) for a, b in ev)
    return [v / 2 for v in sums]


def tune(N: int, M: int, layout: int = 0, bytes_target: int = 3 << 30, reps: int = 5,
         rounds: int = 4, margin: float = 0.01, device: int = 0, sustained_s: float = 0.0):
    """Best launch configuration of sk_flag for (N, M, layout); a dict with the
    sk_launch_config_t fields, the measured table and the chosen one's GB/s.
    sustained_s > 0: each configuration timed over that many seconds of back-to-back
    launches instead of short round-robin rounds."""
    import torch

    dev = torch.device("cuda", device)
    F = max(1, bytes_target // (N * M))
    g = torch.Generator(device=dev)
    g.manual_seed(N * 7919 + M * 31 + layout)
    x = torch.randint(0, 256, (F * N * M,), dtype=torch.uint8, device=dev, generator=g)
    sk = torch.empty(F, dtype=torch.float32, device=dev)
    mask = torch.empty(F, dtype=torch.uint8, device=dev)
    plans = []
    try:
        probe = sk_plan_create(N, M, layout=layout, device=device)
        plans.append(probe)
        # the plan's own input-major team size (0 without an input-major fast path)
        team0 = sk_plan_get_config(probe)["team_log2"]
        cands = candidates(N, M, layout, team0)
        fns, taken = [], []
        for c in cands:
            p = sk_plan_create(N, M, layout=layout, device=device)
            plans.append(p)
            sk_plan_set_config(p, **c)
            fns.append(lambda p=p: sk_flag(p, x, F, sk, mask))
        if sustained_s > 0:
            est = _time_round_robin(fns[:1], 2, 1)[0]
            ms = _time_sustained(fns, sustained_s, est)
        else:
            ms = _time_round_robin(fns, reps, rounds)
        for p in plans[1:]:
            taken.append(sk_plan_get_config(p)["last_path"])
    finally:
        for p in plans:
            sk_plan_destroy(p)
    table = [dict(c, ms=m, gbs=F * N * M / m / 1e6, taken=PATH_NAMES[t])
             for c, m, t in zip(cands, ms, taken)]
    best = min(range(len(ms)), key=lambda k: ms[k])
    if ms[best] > ms[0] * (1.0 - margin):
        best = 0
    out = {k: cands[best][k] for k in FIELDS}
    out.update(N=N, M=M, layout=layout, ms=ms[best], gbs=F * N * M / ms[best] / 1e6,
               default_gbs=F * N * M / ms[0] / 1e6, table=table, sustained_s=sustained_s)
    if layout == 0 and N == 2048 and M % 32 == 0 and sustained_s <= 0:
        out["batch_path"], out["batch_table"] = tune_batch_path(N, M, device=device,
                                                                 reps=reps, rounds=rounds,
                                                                 margin=margin)
    return out


def tune_batch_path(N: int, M: int, bytes_target: int = 3 << 30, reps: int = 5,
                    rounds: int = 4, margin: float = 0.01, device: int = 0):
    """The shape's items in a batched launch: team class against warp-slice class,
    on a batch of 8 items of about bytes_target / 8 each."""
    import torch

    dev = torch.device("cuda", device)
    per = max(1, bytes_target // (8 * N * M))
    g = torch.Generator(device=dev)
    g.manual_seed(N * 104729 + M)
    bufs = [torch.randint(0, 256, (per * N * M,), dtype=torch.uint8, device=dev, generator=g)
            for _ in range(8)]
    outs = [(torch.empty(per, dtype=torch.float32, device=dev),
             torch.empty(per, dtype=torch.uint8, device=dev)) for _ in range(8)]
    choices = (SK_PATH_AUTO, SK_PATH_TEAM, SK_PATH_WARP_SLICE)
    plans, batches, fns = [], [], []
    try:
        for bp in choices:
            p = sk_plan_create(N, M, device=device)
            plans.append(p)
            sk_plan_set_config(p, rows=16, batch_path=bp)
            b = sk_batch_create([(p, x, per, s, m) for x, (s, m) in zip(bufs, outs)], device)
            batches.append(b)
            fns.append(lambda b=b: sk_batch_run(b))
        ms = _time_round_robin(fns, reps, rounds)
    finally:
        for b in batches:
            sk_batch_destroy(b)
        for p in plans:
            sk_plan_destroy(p)
    table = [dict(batch_path=PATH_NAMES[c], ms=m, gbs=8 * per * N * M / m / 1e6)
             for c, m in zip(choices, ms)]
    best = min(range(len(ms)), key=lambda k: ms[k])
    if ms[best] > ms[0] * (1.0 - margin):
        best = 0
    return choices[best], table


def cache_line(e) -> str:
    return (f"{e['N']} {e['M']} {e['layout']} {e['rows']} {e['grid_ctas']} {e['path']} "
            f"{e['team_log2']} {e['prefetch']} {e['batch_path']}\n")


def write_cache(path: str, entries):
    """Merge entries into the cache file: a shape's new line replaces its old one."""
    lines = []
    if os.path.exists(path):
        with open(path) as f:
            lines = [ln for ln in f if ln.strip() and not ln.startswith("#")]
    keys = {(str(e["N"]), str(e["M"]), str(e["layout"])) for e in entries}
    keep = [ln for ln in lines if tuple(ln.split()[:3]) not in keys]
    with open(path, "w") as f:
        f.write("# N M layout rows grid path team_log2 prefetch batch_path "
                "(sk_launch_config_t; path 0 auto, 1 team, 2 warp-slice, 3 row-balanced, "
                "6 stream)\n")
        f.writelines(keep)
        for e in entries:
            f.write(cache_line(e))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--json", help="also write every measured configuration here")
    ap.add_argument("--sustained", type=float, default=0.0,
                    help="time each configuration over this many seconds of back-to-back "
                         "launches (the power-capped regime of continuous streaming)")
    ap.add_argument("shapes", nargs="+", help="N:M or N:M:layout")
    a = ap.parse_args(argv)
    entries = []
    for s in a.shapes:
        v = [int(t) for t in s.split(":")]
        N, M, layout = v[0], v[1], v[2] if len(v) > 2 else 0
        e = tune(N, M, layout, sustained_s=a.sustained)
        print(f"N={N} M={M} layout={layout}: path={PATH_NAMES[e['path']]} rows={e['rows']} "
              f"team_log2={e['team_log2']} prefetch={e['prefetch']} "
              f"batch_path={PATH_NAMES[e['batch_path']]}: {e['gbs']:.0f} GB/s "
              f"(default {e['default_gbs']:.0f})", flush=True)
        entries.append(e)
    write_cache(a.out, entries)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(entries, f, indent=1)


if __name__ == "__main__":
    main()
