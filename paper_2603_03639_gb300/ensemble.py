"""Ensemble sharding across GPUs (one process per GPU).

The ensemble average of Sec. II is over independent noise realisations, so
rank r of R evaluates samples s = r*M_local .. (r+1)*M_local - 1 of the global
ensemble on its own GPU, and the ranks meet once per evaluation: an all-reduce
of [F_r, dF_r/du] (1 + K*C*N doubles), divided by R.

The global noise stream is the counter-based SplitMix64 of ``tnrc_sample_noise``:
draw i of seed S is mix(S + (i + 1) * 0x9E3779B97F4A7C15).  Starting the
counter of rank r at offset D is the same as using the seed
S + D * 0x9E3779B97F4A7C15 (mod 2^64), so a rank draws exactly its slice of
the global J with an ordinary ``sample_noise`` call.
"""
_GAMMA = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1


def shard_seed(seed: int, rank: int, m_local: int, n_sites: int, dist: int, terms: int = 1) -> int:
    """Seed whose J[M_local][N-1](x terms) draw equals rows rank*m_local .. of
    the global J drawn from ``seed`` (uniform: one counter per entry; normal:
    two)."""
    per_sample = (n_sites - 1) * terms * (1 if dist == 0 else 2)
    return (seed + rank * m_local * per_sample * _GAMMA) & _MASK


def allreduce_mean(F, grad, group=None):
    """In place: F and grad (torch tensors on the rank's device, or CPU for
    gloo) become the mean over ranks.  One collective of 1 + grad.numel()
    doubles."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    buf = torch.cat([F.reshape(1), grad.reshape(-1)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    buf /= world
    F.reshape(1).copy_(buf[:1])
    grad.reshape(-1).copy_(buf[1:])
    return F, grad
