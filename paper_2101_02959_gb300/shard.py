"""Subdomain sharding over ranks: the host-side exchange and reduction logic of a
Krylov iteration split across GPUs (the paper's own distribution of subdomains
over processes, Section 6, done here by blocks of the subdomain batch).

Every quantity of the interface system is a sum over subdomains (Section 4.1:
S_hat = sum_j R_j^T S^(j) R_j; the coarse right-hand side sums the local primal
contributions, Section 4.4), and the subdomains are independent between those
sums.  So a rank that owns a block of subdomains computes their local products
on its GPU and needs, per Krylov iteration:

* one neighbour exchange: the partial interface sums of the dofs it shares with
  other ranks (``ShardPlan.assemble``), added in ascending rank order so that
  every rank holding a dof obtains the same value bit for bit;
* two or three FP64 scalars summed over ranks (``ShardPlan.dot``: each dof is
  counted by its owner, the lowest rank that holds it);
* the coarse right-hand side summed over ranks (``ShardPlan.allreduce``), after
  which every rank solves the replicated coarse problem itself.

The same calls run on CUDA tensors with the NCCL backend and on CPU tensors with
gloo (how the tests drive them).  Only point-to-point send / receive and all-reduce
are used: no device kernel waits on another rank's memory.
"""
from __future__ import annotations

import numpy as np


def block_partition(n_sub, world):
    """Rank of every subdomain: contiguous blocks of the subdomain order (lexicographic
    over the grid of blocks, so a rank holds a slab of the domain), sizes within one."""
    return (np.arange(n_sub, dtype=np.int64) * world) // n_sub


def subdomain_interface_dofs(sub_node_ptr, sub_nodes, sub_nint, iface_nodes):
    """Global interface dofs (2 x interface index + field) of every subdomain, in its local
    interface order, from the plan's index sets (bd_plan_index_sets)."""
    pos = {int(x): k for k, x in enumerate(iface_nodes)}
    out = []
    for j in range(len(sub_nint)):
        nodes = sub_nodes[sub_node_ptr[j] + sub_nint[j]:sub_node_ptr[j + 1]]
        g = np.array([pos[int(x)] for x in nodes], dtype=np.int64)
        out.append(np.stack([2 * g, 2 * g + 1], axis=1).ravel())
    return out


class ShardPlan:
    """What rank ``rank`` of ``world`` holds and exchanges.

    sub_dofs: global interface dofs of every subdomain; n_iface: their number.
    Attributes: ``subs`` (this rank's subdomains), ``touched`` (sorted interface dofs
    they reach), ``owned`` (boolean over ``touched``: this rank is the lowest holder),
    ``shared`` ({peer rank: sorted dofs held by both}).
    """

    def __init__(self, sub_dofs, n_iface, world, rank, part=None):
        self.world, self.rank, self.n_iface = int(world), int(rank), int(n_iface)
        part = block_partition(len(sub_dofs), world) if part is None else np.asarray(part)
        self.part = part
        self.subs = np.flatnonzero(part == rank)
        holders = [set() for _ in range(n_iface)]
        for j, d in enumerate(sub_dofs):
            for g in d:
                holders[int(g)].add(int(part[j]))
        self.touched = np.array(sorted({int(g) for j in self.subs for g in sub_dofs[j]}), dtype=np.int64)
        self.owned = np.array([min(holders[g]) == rank for g in self.touched], dtype=bool)
        self.shared = {}
        for g in self.touched:
            for r in holders[int(g)]:
                if r != rank:
                    self.shared.setdefault(r, []).append(int(g))
        self.shared = {r: np.array(v, dtype=np.int64) for r, v in sorted(self.shared.items())}

    # -- collectives (torch.distributed; CPU tensors with gloo, CUDA tensors with NCCL) --
    def assemble(self, partial):
        """Interface assembly across ranks: ``partial`` is a full-length vector (torch,
        float64) holding this rank's subdomain sums on ``touched``.  Returns the global
        sums on ``touched`` (zero elsewhere), identical on every rank holding a dof."""
        import torch
        import torch.distributed as dist
        recv, reqs = {}, []
        for peer, dofs in self.shared.items():
            idx = torch.as_tensor(dofs, device=partial.device)
            send = partial.index_select(0, idx).contiguous()
            buf = torch.empty_like(send)
            recv[peer] = (idx, buf)
            # the lower rank sends first, so that every pair of blocking calls matches
            if self.rank < peer:
                dist.send(send, peer)
                dist.recv(buf, peer)
            else:
                dist.recv(buf, peer)
                dist.send(send, peer)
        out = torch.zeros_like(partial)
        mine = torch.as_tensor(self.touched, device=partial.device)
        for r in range(self.world):  # fixed (ascending rank) order of the additions
            if r == self.rank:
                out.index_add_(0, mine, partial.index_select(0, mine))
            elif r in recv:
                idx, buf = recv[r]
                out.index_add_(0, idx, buf)
        return out

    def dot(self, a, b):
        """sum over all interface dofs of a b, each counted once (by its owner rank)."""
        import torch
        import torch.distributed as dist
        idx = torch.as_tensor(self.touched[self.owned], device=a.device)
        s = (a.index_select(0, idx) * b.index_select(0, idx)).sum().reshape(1).to(torch.float64)
        dist.all_reduce(s)
        return float(s.item())

    def allreduce(self, v):
        """Sum of a vector over ranks (the coarse right-hand side before the replicated
        coarse solve)."""
        import torch.distributed as dist
        v = v.clone()
        dist.all_reduce(v)
        return v
