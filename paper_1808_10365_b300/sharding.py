"""Input sharding: the inputs of one frequency spread over the ranks of a process
group, one GPU each.  The per-input terms of Eq. final depend on their own input
only, so a frame's fixed-point sum Q and its N_eff are the exact integer sums of
the ranks' values: one all-reduce of 12 bytes a frame is the whole exchange, and
the result is bit-identical to flagging the whole array on one device.

Each rank holds its own inputs' bytes as one contiguous array ([frame][t][input]
or [frame][input][t], as its plan says) and a plan for them (its own N), plus the
plan of the whole array (N = the total, same M, sigma and offset) for the
thresholds.  Argument marshalling and the collective only: S1, S2, the terms, Q
and the mask are formed by the library's kernels."""

from __future__ import annotations

import paper_1808_10365_b300 as sk


def exchange_partials(q, neff, group=None):
    """Sum per-frame Q (int64) and N_eff (int32) over the ranks in place: exact
    integer all-reduces (NCCL for CUDA tensors, gloo for CPU tensors)."""
    import torch.distributed as dist

    dist.all_reduce(q, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(neff, op=dist.ReduceOp.SUM, group=group)
    return q, neff


def flag_sharded(plan_shard, plan_all, d_in, n_frames, d_sk, d_mask, group=None, stream=None):
    """SK and mask of n_frames frames whose inputs are spread over the group's
    ranks: this rank's Q and N_eff (sk_compute on its shard), their sums over the
    group, then sk_finish with the whole array's plan.  d_sk may be None.  With
    a stream, the three steps are ordered on it (the collective waits for the
    stream's work, as torch.distributed does for the current stream)."""
    import contextlib

    import torch

    dev = d_mask.device
    F = int(n_frames)
    ctx = torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()
    with ctx:
        q = torch.empty(max(F, 1), dtype=torch.int64, device=dev)
        neff = torch.empty(max(F, 1), dtype=torch.int32, device=dev)
        sk.sk_compute(plan_shard, d_in, F, None, None, q, None, neff, stream)
        exchange_partials(q[:F], neff[:F], group)
        sk.sk_finish(plan_all, q, neff, F, d_sk, d_mask, stream)
    return q[:F], neff[:F]
