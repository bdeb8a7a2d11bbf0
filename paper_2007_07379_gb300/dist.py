"""Multi-rank sharding of the chains and the one exchange of the method.

Chains are independent Markov chains (Fig. 2 runs one per sample stream), so
rank r of R owns a contiguous range of 32-chain groups; its draws depend on
the global group index only (pb_run_cfg.group0), so the union of the ranks'
chains is exactly the single-process run.  The only exchange is the integer
sum of the histograms and counters after the sweeps (exact, order
independent); models with general gates add their FP64 phase sums (sums of
unit phasors, rounding-level order dependence).
"""
from __future__ import annotations

import numpy as np


def shard(chains: int, rank: int, world: int) -> tuple[int, int]:
    """(chains on this rank, first global group) for `chains` chains split
    over `world` ranks by whole 32-chain groups (earlier ranks take the
    remainder)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    groups = (chains + 31) // 32
    base, extra = divmod(groups, world)
    g0 = rank * base + min(rank, extra)
    g = base + (1 if rank < extra else 0)
    first_chain = g0 * 32
    last_chain = min(chains, (g0 + g) * 32)
    return max(0, last_chain - first_chain), g0


def allreduce_histogram(counts: np.ndarray, valid: int, samples: int, device=None):
    """Integer sum over ranks of (counts[bins, 8], valid, samples) with
    torch.distributed (gloo on CPU tensors, NCCL on CUDA tensors)."""
    import torch
    import torch.distributed as dist
    flat = np.concatenate([np.asarray(counts, dtype=np.uint64).reshape(-1),
                           np.array([valid, samples], dtype=np.uint64)]).astype(np.int64)
    t = torch.from_numpy(flat)
    if device is not None:
        t = t.to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    out = t.cpu().numpy().astype(np.uint64)
    return out[:-2].reshape(np.asarray(counts).shape), int(out[-2]), int(out[-1])


def allreduce_phase_sums(sums: np.ndarray, counts: np.ndarray, valid: int, samples: int,
                         device=None):
    """Sum over ranks of a general-gate model's phase sums (complex[bins],
    FP64) and of its integer counters (counts[bins], valid, samples; exact)."""
    import torch
    import torch.distributed as dist
    ints = np.concatenate([np.asarray(counts, dtype=np.uint64).reshape(-1),
                           np.array([valid, samples], dtype=np.uint64)]).astype(np.int64)
    z = np.asarray(sums, dtype=np.complex128).reshape(-1)
    flo = np.concatenate([z.real, z.imag])
    ti, tf = torch.from_numpy(ints), torch.from_numpy(flo)
    if device is not None:
        ti, tf = ti.to(device), tf.to(device)
    dist.all_reduce(ti, op=dist.ReduceOp.SUM)
    dist.all_reduce(tf, op=dist.ReduceOp.SUM)
    oi = ti.cpu().numpy().astype(np.uint64)
    of = tf.cpu().numpy()
    b = z.size
    return (of[:b] + 1j * of[b:]).reshape(np.asarray(sums).shape), \
        oi[:-2].reshape(np.asarray(counts).shape), int(oi[-2]), int(oi[-1])
