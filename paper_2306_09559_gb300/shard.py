"""Noise sharding across processes (one process per GPU).

The noise vectors of a level are independent: the Philox counter of noise j
is the global index j, so a sample does not depend on which process draws
it.  Rank r of P takes a contiguous range of noise indices, computes its
samples with the same block width as a single process would (so they are
bit-identical to the single-process ones), and one exchange step gathers the
FP64 per-sample values on rank 0 in global-j order.  The statistics are then
formed on rank 0 exactly as for one process.  There is no halo exchange and
no collective inside a level's computation.
"""

import numpy as np


def partition(nsamples, world, rank):
    """(first, count) of rank's contiguous share of noise indices 0 .. nsamples-1."""
    if world < 1 or not 0 <= rank < world or nsamples < 0:
        raise ValueError("bad partition arguments")
    base, extra = divmod(nsamples, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def level_statistics(samples):
    """Per level: mean of the complex samples and sample variance of their real
    parts (N - 1 in the denominator), summed in index order."""
    L, N = samples.shape
    mean = np.zeros(L, dtype=np.complex128)
    var = np.full(L, np.nan)
    for l in range(L):
        mr = mi = 0.0
        for z in samples[l]:
            mr += float(z.real)
            mi += float(z.imag)
        mr /= N
        mi /= N
        mean[l] = complex(mr, mi)
        if N > 1:
            v = 0.0
            for z in samples[l]:
                d = float(z.real) - mr
                v += d * d
            var[l] = v / (N - 1)
    return mean, var


def gather_samples(local, nsamples, group=None):
    """Gather every rank's (L, count) complex samples on rank 0 in global-j order.

    local: this rank's samples for partition(nsamples, world, rank).  Returns
    the (L, nsamples) array on rank 0 and None elsewhere.  Works with any
    torch.distributed backend that gathers CPU tensors (gloo) or device
    tensors (nccl, after moving them there).
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    L = local.shape[0]
    counts = [partition(nsamples, world, r)[1] for r in range(world)]
    width = max(counts) if counts else 0
    buf = np.zeros((L, width, 2), dtype=np.float64)
    buf[:, :local.shape[1], 0] = local.real
    buf[:, :local.shape[1], 1] = local.imag
    mine = torch.from_numpy(buf)
    backend = dist.get_backend(group)
    if backend == "nccl":
        mine = mine.cuda()
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    if rank != 0:
        return None
    out = np.empty((L, nsamples), dtype=np.complex128)
    for r, p in enumerate(parts):
        first, cnt = partition(nsamples, world, r)
        a = p.cpu().numpy()
        out[:, first:first + cnt] = a[:, :cnt, 0] + 1j * a[:, :cnt, 1]
    return out


def sharded_trace(compute, nsamples, group=None):
    """Run compute(first, count) -> (L, count) samples on this rank's share and
    gather on rank 0.  Returns (samples, mean, var) on rank 0, None elsewhere;
    the caller adds each level's exact deflation correction to the mean."""
    import torch.distributed as dist
    first, count = partition(nsamples, dist.get_world_size(group), dist.get_rank(group))
    local = np.asarray(compute(first, count), dtype=np.complex128)
    allv = gather_samples(local, nsamples, group)
    if allv is None:
        return None
    mean, var = level_statistics(allv)
    return allv, mean, var
