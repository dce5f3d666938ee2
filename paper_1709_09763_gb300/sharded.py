"""Particle sharding across ranks: the exchange steps of a sampler whose J particles are split over
R processes (one GPU each, `torch.distributed`; NCCL on GPUs, gloo on the host).

Rank r owns the particles with global indices [lo_r, hi_r) (`shard_bounds`: contiguous, sizes
differing by at most one). Every step of an importance-sampling update is local to a particle
(likelihood, Markov moves) except two, which need all J weights:

1. the adaptive increment (Sec. 3.4, Eq. Eq_cv_opt): the cv and the log mean weight are sums
   over all particles. The ranks all-gather the J potentials, or the J incremental
   log-weights of a bridging step (`allgather_rows`, J doubles), and every rank runs the same
   deterministic search on identical inputs, so all ranks take the same increment;
2. systematic resampling (Sec. 2.4): with one offset U drawn from the shared seed, every rank
   computes the same J ancestors from the gathered weights. Output particle i then takes the
   row (theta and its potential caches) of ancestor a(i), which lives on rank owner(a(i)).
   Systematic ancestors are non-decreasing in i, so each (source, destination) pair of ranks
   exchanges one contiguous block of rows (`exchange_plan`); `exchange_rows` moves only rows
   that change rank, with one point-to-point message per pair that has any.

After the exchange every rank again holds the rows of its own output range [lo_r, hi_r), in
order: the concatenation over ranks is the single-rank result. Nothing else crosses ranks. For a
sharded run to use the same random numbers as one process holding all J particles, each rank's
Markov moves must draw from Philox counters that carry the particle's global index (the
library's counter layout has the particle index in its second word; a shard offsets it by lo_r).
"""
import numpy as np


def shard_bounds(J, world):
    """[lo_r, hi_r) for r = 0..world-1: contiguous, the first J % world shards one longer."""
    if J < 0 or world < 1:
        raise ValueError("J >= 0 and world >= 1 required")
    base, extra = divmod(J, world)
    sizes = [base + (1 if r < extra else 0) for r in range(world)]
    lo = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return [(int(lo[r]), int(lo[r + 1])) for r in range(world)]


def owner_of(indices, bounds):
    """Rank that owns each global particle index."""
    starts = np.array([b[0] for b in bounds], dtype=np.int64)
    idx = np.asarray(indices, dtype=np.int64)
    J = bounds[-1][1]
    if idx.size and (idx.min() < 0 or idx.max() >= J):
        raise ValueError("particle index out of range")
    return np.searchsorted(starts, idx, side="right") - 1


def exchange_plan(anc, bounds):
    """For the global ancestor array `anc` [J] (non-decreasing, systematic resampling): the rows
    each rank sends and receives.

    Returns plan[src][dst] = (pos, count): output positions [pos, pos + count) of rank dst (relative
    to its lo) take the rows anc[lo_dst + pos: lo_dst + pos + count], all of which rank src owns.
    Pairs that exchange nothing are absent."""
    anc = np.asarray(anc, dtype=np.int64)
    J = bounds[-1][1]
    if anc.shape != (J,):
        raise ValueError("ancestor array must have J entries")
    if J and np.any(np.diff(anc) < 0):
        raise ValueError("systematic ancestors are non-decreasing")
    world = len(bounds)
    src_of = owner_of(anc, bounds)
    plan = [dict() for _ in range(world)]
    for dst, (lo, hi) in enumerate(bounds):
        if hi == lo:
            continue
        s = src_of[lo:hi]
        # runs of equal source rank inside dst's range (one per source, since s is non-decreasing)
        cut = np.flatnonzero(np.diff(s)) + 1
        starts = np.concatenate([[0], cut])
        ends = np.concatenate([cut, [hi - lo]])
        for a, b in zip(starts, ends):
            plan[int(s[a])][dst] = (int(a), int(b - a))
    return plan


def allgather_rows(local, group=None):
    """All ranks' row blocks (torch tensors, [n_r, ...], n_r from shard_bounds) concatenated in
    rank order on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = torch.tensor([local.shape[0]], dtype=torch.int64, device=local.device)
    all_sizes = [torch.zeros_like(sizes) for _ in range(world)]
    dist.all_gather(all_sizes, sizes, group=group)
    n = [int(x.item()) for x in all_sizes]
    m = max(n) if n else 0
    pad = torch.zeros((m,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:k] for p, k in zip(parts, n)], dim=0)


def exchange_rows(local, anc, bounds, group=None):
    """Rows of this rank's output range after resampling: out[i - lo] = row anc[i] (global),
    taken from the rank that owns it. `local` is this rank's [hi - lo, ...] block before
    resampling; `anc` the global ancestor array that every rank computed identically."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    if len(bounds) != world:
        raise ValueError("bounds must have one entry per rank")
    anc = np.asarray(anc, dtype=np.int64)
    plan = exchange_plan(anc, bounds)
    lo, hi = bounds[rank]
    out = torch.empty((hi - lo,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    reqs, recv = [], []
    for dst, (pos, cnt) in plan[rank].items():          # rows this rank supplies
        rows = torch.as_tensor(anc[bounds[dst][0] + pos: bounds[dst][0] + pos + cnt] - lo, device=local.device)
        block = local.index_select(0, rows)
        if dst == rank:
            out[pos:pos + cnt] = block
        else:
            reqs.append(dist.isend(block.contiguous(), dst, group=group))
    for src in range(world):                              # rows this rank receives
        if src == rank or rank not in plan[src]:
            continue
        pos, cnt = plan[src][rank]
        buf = torch.empty((cnt,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
        reqs.append(dist.irecv(buf, src, group=group))
        recv.append((pos, cnt, buf))
    for r in reqs:
        r.wait()
    for pos, cnt, buf in recv:
        out[pos:pos + cnt] = buf
    return out
