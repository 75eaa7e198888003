"""Autotuner for the fused kernel's tile choice.

For each (N, M) class it times sk_flag over a device-resident batch for every
rows-per-batch (8, 16) and a few grid sizes, and writes the fastest to the
cache file that sk_plan_create reads (environment variable SK_AUTOTUNE_CACHE;
lines "N M layout rows grid").  Results never depend on the tiles (exact
integer combination), only speed does.  Input bytes are uniform random: the
kernel's cost does not depend on their values.

    python -m paper_1808_10365_b300.autotune --out sk_tiles.txt 2048:256 256:256
"""

from __future__ import annotations

import argparse
import os

from . import (sk_flag, sk_plan_create, sk_plan_destroy, sk_plan_set_tiles)


def tune(N: int, M: int, bytes_target: int = 1 << 30, reps: int = 10, device: int = 0):
    import torch

    dev = torch.device("cuda", device)
    F = max(1, bytes_target // (N * M))
    g = torch.Generator(device=dev)
    g.manual_seed(N * 7919 + M)
    x = torch.randint(0, 256, (F * N * M,), dtype=torch.uint8, device=dev, generator=g)
    sk = torch.empty(F, dtype=torch.float32, device=dev)
    mask = torch.empty(F, dtype=torch.uint8, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    plan = sk_plan_create(N, M, device=device)
    results = []
    try:
        for rows in (8, 16):
            for grid in (0, sms // 2, 2 * sms):
                sk_plan_set_tiles(plan, rows, grid)
                for _ in range(2):
                    sk_flag(plan, x, F, sk, mask)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(reps):
                    sk_flag(plan, x, F, sk, mask)
                b.record()
                torch.cuda.synchronize()
                ms = a.elapsed_time(b) / reps
                results.append((ms, rows, grid))
    finally:
        sk_plan_destroy(plan)
    results.sort()
    ms, rows, grid = results[0]
    return dict(N=N, M=M, rows=rows, grid=grid, ms=ms, gbs=F * N * M / ms / 1e6, all=results)


def write_cache(path: str, entries):
    lines = []
    if os.path.exists(path):
        with open(path) as f:
            lines = [ln for ln in f if ln.strip() and not ln.startswith("#")]
    keep = [ln for ln in lines
            if not any(ln.split()[:3] == [str(e["N"]), str(e["M"]), "0"] for e in entries)]
    with open(path, "w") as f:
        f.write("# N M layout rows grid (fused SK kernel tiles)\n")
        f.writelines(keep)
        for e in entries:
            f.write(f"{e['N']} {e['M']} 0 {e['rows']} {e['grid']}\n")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("shapes", nargs="+", help="N:M pairs")
    a = ap.parse_args(argv)
    entries = []
    for s in a.shapes:
        N, M = (int(v) for v in s.split(":"))
        e = tune(N, M)
        print(f"N={N} M={M}: rows={e['rows']} grid={e['grid']} {e['gbs']:.0f} GB/s", e["all"])
        entries.append(e)
    write_cache(a.out, entries)


if __name__ == "__main__":
    main()
