"""A multilevel estimate spread over several processes, one per GPU.

The probes of the multilevel estimator are independent samples (Section 4,
Eq. multiEstimator), so a run shards by probe ids with two small exchanges:

  1. Rank 0 runs the pilot (probe ids 0 .. m_pilot-1 at degree n), its variance
     table and the level selection (Section 3.2.1, Theorem levels, Eqs.
     optSamples / optMu) and broadcasts the levels, the sample counts and the
     top band of the pilot rows (those rows are the top level's first samples).
  2. The fresh probes run level by level from id m_pilot on, exactly as
     mlt_mlmc_estimate numbers them.  Rank r takes the r-th contiguous part of
     that id sequence, computes the moments of its part in one ragged call and
     turns each row into its level's band sample Q_{l_{k-1} l_k}.
  3. The band samples (one double per probe) are gathered to every rank in rank
     order, which is probe-id order, and combined.

Every arithmetic step is the library's (mlt_pilot_variances,
mlt_select_levels, mlt_band_samples, mlt_mlmc_combine; the same routines
mlt_mlmc_estimate calls), and the moments come from the caller's moment
function, normally `library_moments` (mlt_moments on this rank's GPU).  So with
the same moments for the same probe ids, a run on any number of ranks combines
the same samples in the same order as one process does, to the last bit.
torch.distributed only moves the plan and the samples: NCCL with CUDA tensors,
gloo with host tensors.
"""
from __future__ import annotations

import numpy as np

from . import mlt


def split_range(count, rank, world):
    """[start, start + size) of rank's contiguous part of `count` items: the
    first count % world ranks take one item more."""
    base, rem = divmod(int(count), int(world))
    start = rank * base + min(rank, rem)
    return start, base + (1 if rank < rem else 0)


def library_moments(handle, a, b, seed, precision="fp64", flags=0, stream=None):
    """Moment function over the library: (probe_offset, degrees) -> host rows."""
    def f(probe_offset, degrees):
        return mlt.mlt_moments(handle, a, b, seed, probe_offset, degrees, precision=precision, flags=flags,
                               stream=stream)
    return f


def _fresh_plan(levels, m, m_pilot, reuse_pilot):
    fresh = list(m)
    if m_pilot > 0 and reuse_pilot:
        fresh[-1] = m[-1] - m_pilot
    deg = np.concatenate([np.full(f, l, dtype=np.int32) for l, f in zip(levels, fresh)]) \
        if sum(fresh) else np.zeros(0, dtype=np.int32)
    lev = np.concatenate([np.full(f, k, dtype=np.int32) for k, f in enumerate(fresh)]) \
        if sum(fresh) else np.zeros(0, dtype=np.int32)
    return fresh, deg, lev


def _samples_of(c, levels, lev, mu):
    """Band sample of each moment row, row p on level lev[p]."""
    q = np.zeros(lev.size)
    for k in np.unique(lev):
        rows = np.nonzero(lev == k)[0]
        lo = levels[k - 1] if k > 0 else -1
        q[rows] = mlt.mlt_band_samples(c, lo, levels[k], mu[rows])
    return q


def mlmc_sharded(moments, fn, a, b, n, m_pilot=10, mode="budget", target=1000.0, cost_model="symmetric",
                 max_levels=0, reuse_pilot=True, levels=None, m=None, p=0.0, group=None, direct=False):
    """Multilevel estimate of tr p_n(At) with the work of every level split over
    the ranks of `group` (torch.distributed; None or a single process: no
    collectives).  `moments(probe_offset, degrees)` returns the host moment rows
    (nprobes x (max degree + 1)) of the probes with ids probe_offset + i.
    Fixed levels and sample counts (`levels`, `m`) skip the pilot.  Returns the
    dict of mlt_mlmc_estimate; `matvecs` counts every rank's operator
    applications, ceil(l/2) per probe of degree l with the doubling evaluation
    or l when the moments run direct (MLT_DIRECT), as mlt_mlmc_estimate does."""
    world, rank, dist = 1, 0, None
    if group is not None or _dist_ready():
        import torch.distributed as dist
        world = dist.get_world_size(group)
        rank = dist.get_rank(group)
        if world == 1:
            dist = None
    c = mlt.mlt_cheb_coeffs(fn, a, b, n, p)
    steps = (lambda l: l) if direct else (lambda l: (l + 1) // 2)
    # 1. plan: levels, counts and the pilot's top-band samples (rank 0)
    if levels is not None:
        levels = [int(v) for v in levels]
        m = [int(v) for v in m]
        m_pilot_used = 0
        top_pilot = np.zeros(0)
    else:
        m_pilot_used = int(m_pilot)
        top_pilot = np.zeros(0)
        if rank == 0:
            pilot = moments(0, np.full(m_pilot_used, n, dtype=np.int32))
            V = mlt.mlt_pilot_variances(c, pilot)
            levels, m = mlt.mlt_select_levels(V, cost_model, m_pilot_used if reuse_pilot else 0, mode, target,
                                              max_levels)
            lo = levels[-2] if len(levels) > 1 else -1
            top_pilot = mlt.mlt_band_samples(c, lo, n, pilot) if reuse_pilot else np.zeros(0)
        if dist is not None:
            levels, m, top_pilot = _broadcast_plan(dist, group, rank, levels, m, top_pilot)
    fresh, deg, lev = _fresh_plan(levels, m, m_pilot_used, reuse_pilot)
    # 2. this rank's contiguous part of the fresh id sequence
    first_id = m_pilot_used
    start, size = split_range(deg.size, rank, world)
    if size > 0:
        mu = np.asarray(moments(first_id + start, deg[start:start + size]), dtype=np.float64)
        q = _samples_of(c, levels, lev[start:start + size], mu)
    else:
        q = np.zeros(0)
    # 3. every rank's samples, in rank (= probe id) order
    if dist is not None:
        q_all = _all_gather_parts(dist, group, q, [split_range(deg.size, r, world)[1] for r in range(world)])
    else:
        q_all = q
    # Eq. multiEstimator: level by level, the pilot rows first on a reusing top level
    L = len(levels)
    offs = np.concatenate([[0], np.cumsum(fresh)])
    parts = []
    for k in range(L):
        if k == L - 1 and top_pilot.size:
            parts.append(top_pilot)
        parts.append(q_all[offs[k]:offs[k + 1]])
    out = mlt.mlt_mlmc_combine(levels, m, np.concatenate(parts) if parts else np.zeros(0))
    out["probes"] = first_id + int(deg.size)
    out["matvecs"] = int(m_pilot_used * steps(n) + sum(int(f) * steps(l) for l, f in zip(levels, fresh)))
    out["ranks"] = world
    return out


def _dist_ready():
    try:
        import torch.distributed as dist
        return dist.is_available() and dist.is_initialized()
    except Exception:
        return False


def _device(dist, group):
    import torch
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")


def _broadcast_plan(dist, group, rank, levels, m, top_pilot):
    """Rank 0's levels, counts and pilot top-band samples to every rank (the
    counts are exact in float64 far beyond any sample count)."""
    import torch
    dev = _device(dist, group)
    head = torch.zeros(2, dtype=torch.float64, device=dev)
    if rank == 0:
        head[0] = len(levels)
        head[1] = len(top_pilot)
    dist.broadcast(head, src=dist.get_global_rank(group, 0) if group is not None else 0, group=group)
    L, P = int(head[0].item()), int(head[1].item())
    body = torch.zeros(2 * L + P, dtype=torch.float64, device=dev)
    if rank == 0:
        body.copy_(torch.from_numpy(np.concatenate([np.asarray(levels, dtype=np.float64),
                                                    np.asarray(m, dtype=np.float64),
                                                    np.asarray(top_pilot, dtype=np.float64)])))
    dist.broadcast(body, src=dist.get_global_rank(group, 0) if group is not None else 0, group=group)
    b = body.cpu().numpy()
    return [int(v) for v in b[:L]], [int(v) for v in b[L:2 * L]], b[2 * L:].copy()


def _all_gather_parts(dist, group, q, sizes):
    """Concatenation of every rank's samples (rank order), parts padded to the
    largest for the collective."""
    import torch
    dev = _device(dist, group)
    w = max(max(sizes), 1)
    mine = torch.zeros(w, dtype=torch.float64, device=dev)
    if q.size:
        mine[:q.size] = torch.from_numpy(q).to(dev)
    bufs = [torch.zeros(w, dtype=torch.float64, device=dev) for _ in sizes]
    dist.all_gather(bufs, mine, group=group)
    return np.concatenate([bufs[r][:sizes[r]].cpu().numpy() for r in range(len(sizes))])
