"""Halo exchange of a split box by its plan (grf_halo_plan), on one process or across the ranks
of a torch.distributed group.

The plan lists rectangular blocks: ghost points of patch `dst` that equal interior points of
patch `src` (all 27 fields). Applying every block fills every ghost point the built-in device
exchange (grf_halo_exchange) fills, with the same values. Across ranks, each rank holds the
states of the patches it owns; a block whose source and destination live on different ranks is
packed by the source's rank, sent point to point (send/recv into the receiving rank's own
buffer) and unpacked into the destination patch. With the gloo backend the states are CPU
tensors; with NCCL they are device tensors of each rank's own GPU.
"""
from __future__ import annotations


def _region(state, k0, j0, i0, nk, nj, ni):
    return state[:, k0:k0 + nk, j0:j0 + nj, i0:i0 + ni]


def apply_plan(plan, patches):
    """Copies every block of the plan among the given patch states (all patches local; numpy
    arrays or torch tensors of shape (27, nz + 6, ny + 6, pitch))."""
    for b in plan:
        src = _region(patches[b.src], b.src_k, b.src_j, b.src_i, b.nk, b.nj, b.ni)
        dst = _region(patches[b.dst], b.dst_k, b.dst_j, b.dst_i, b.nk, b.nj, b.ni)
        dst[...] = src


def exchange(plan, local, owner, rank, group=None):
    """One exchange across ranks. local: {patch index: tensor} of the patches this rank owns;
    owner[q]: the rank owning patch q. Blocks between two local patches are copied directly;
    the others are sent by the source's rank and received by the destination's, matched by the
    block's position in the plan (the tag). Returns when every receive has completed."""
    import torch
    import torch.distributed as dist
    sends, recvs = [], []
    for tag, b in enumerate(plan):
        s_own, d_own = owner[b.src], owner[b.dst]
        if s_own == rank and d_own == rank:
            _region(local[b.dst], b.dst_k, b.dst_j, b.dst_i, b.nk, b.nj, b.ni)[...] = \
                _region(local[b.src], b.src_k, b.src_j, b.src_i, b.nk, b.nj, b.ni)
        elif s_own == rank:
            buf = _region(local[b.src], b.src_k, b.src_j, b.src_i, b.nk, b.nj, b.ni).contiguous()
            sends.append((dist.isend(buf, dst=d_own, group=group, tag=tag), buf))
        elif d_own == rank:
            t = local[b.dst]
            buf = torch.empty((t.shape[0], b.nk, b.nj, b.ni), dtype=t.dtype, device=t.device)
            recvs.append((dist.irecv(buf, src=s_own, group=group, tag=tag), b, buf))
    for req, b, buf in recvs:
        req.wait()
        _region(local[b.dst], b.dst_k, b.dst_j, b.dst_i, b.nk, b.nj, b.ni)[...] = buf
    for req, _ in sends:
        req.wait()
