"""Spatial domain decomposition of one system over ranks: the host-side halo
logic of the multi-GPU design (the paper's MPI fix exchanged ghost-atom
electronic temperatures every substep, Sec. 2.1 and Sec. 3.2 scaling).

A rank owns the atoms of a slab along one axis.  Its local system is its owned
atoms plus the ghosts: the atoms of other ranks that are neighbours of an owned
atom.  Local ids follow ascending original ids, so every owned atom's neighbour
row keeps the order of the global list, and a Jacobi substep on the local system
gives the owned atoms exactly the values of the undivided system.  Before every
substep each rank sends the current values of its owned atoms that other ranks
hold as ghosts and overwrites its ghosts with what it receives.

This module holds no arithmetic of the method: it partitions, plans and moves
values; the substep itself is the caller's (one context per rank)."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def slab_owner(x: np.ndarray, box, n_ranks: int, axis: int = 0) -> np.ndarray:
    """Owning rank of every atom: n_ranks equal slabs of the box along `axis`."""
    L = float(box[axis])
    r = np.floor(np.asarray(x)[:, axis] / L * n_ranks).astype(np.int64)
    return np.clip(r, 0, n_ranks - 1)


@dataclass
class HaloPlan:
    """One rank's local system and its exchange lists (all ids original unless
    named local)."""
    rank: int
    local_ids: np.ndarray            # original ids of the local atoms, ascending
    n_owned: int
    owned_mask: np.ndarray           # [n_local] True for owned atoms
    rowptr: np.ndarray               # local neighbour list: owned rows as in the global list, ghost rows empty
    col: np.ndarray                  # local ids
    send: dict = field(default_factory=dict)   # peer -> local ids of owned atoms the peer holds as ghosts
    recv: dict = field(default_factory=dict)   # peer -> local ids of ghosts owned by the peer (peer's send order)


def plan(rowptr: np.ndarray, col: np.ndarray, owner: np.ndarray, rank: int) -> HaloPlan:
    """The local system of `rank` from the global neighbour list."""
    n = owner.shape[0]
    owned = np.flatnonzero(owner == rank)
    cnt = rowptr[owned + 1] - rowptr[owned]
    idx = np.repeat(rowptr[owned] - np.cumsum(cnt) + cnt, cnt) + np.arange(int(cnt.sum()))
    nb = col[idx]
    ghosts = np.unique(nb[owner[nb] != rank])
    local = np.union1d(owned, ghosts)                 # ascending original ids
    loc = -np.ones(n, dtype=np.int64)
    loc[local] = np.arange(local.size)
    is_owned = owner[local] == rank
    lcnt = np.zeros(local.size, dtype=np.int64)
    lcnt[loc[owned]] = cnt
    lrowptr = np.concatenate([[0], np.cumsum(lcnt)]).astype(np.int64)
    lcol = np.empty(int(lcnt.sum()), dtype=np.int32)
    # rows of owned atoms, in local order, each as in the global list
    pos = 0
    order = np.argsort(loc[owned])
    for i in owned[order]:
        a, b = rowptr[i], rowptr[i + 1]
        lcol[pos:pos + (b - a)] = loc[col[a:b]]
        pos += b - a
    p = HaloPlan(rank=rank, local_ids=local, n_owned=int(owned.size), owned_mask=is_owned,
                 rowptr=lrowptr, col=lcol)
    # ghosts held here, grouped by owner (ascending original id within a peer)
    for q in np.unique(owner[ghosts]):
        g = ghosts[owner[ghosts] == q]
        p.recv[int(q)] = loc[g]
    return p


def link_sends(plans: list[HaloPlan]) -> None:
    """Fill every plan's send lists from the peers' ghost lists (all plans known:
    the single-process form; `exchange_plan` does it over torch.distributed)."""
    for p in plans:
        for q in plans:
            if q.rank == p.rank or p.rank not in q.recv:
                continue
            ghost_orig = q.local_ids[q.recv[p.rank]]
            p.send[q.rank] = np.searchsorted(p.local_ids, ghost_orig)


def exchange_plan(p: HaloPlan, dist) -> None:
    """Tell every peer which of its atoms this rank holds as ghosts (original ids),
    and fill this rank's send lists from what the peers ask for."""
    import torch
    ws = dist.get_world_size()
    for q in range(ws):
        if q == p.rank:
            continue
        want = torch.as_tensor(p.local_ids[p.recv[q]] if q in p.recv else np.zeros(0, np.int64), dtype=torch.int64)
        n_want = torch.tensor([want.numel()], dtype=torch.int64)
        n_ask = torch.zeros(1, dtype=torch.int64)
        # the lower rank sends first, so the pairs never wait on each other
        if p.rank < q:
            dist.send(n_want, q)
            dist.recv(n_ask, q)
        else:
            dist.recv(n_ask, q)
            dist.send(n_want, q)
        ask = torch.zeros(int(n_ask.item()), dtype=torch.int64)
        if p.rank < q:
            if want.numel():
                dist.send(want, q)
            if ask.numel():
                dist.recv(ask, q)
        else:
            if ask.numel():
                dist.recv(ask, q)
            if want.numel():
                dist.send(want, q)
        if ask.numel():
            p.send[q] = np.searchsorted(p.local_ids, ask.numpy())


def exchange_values(p: HaloPlan, values: np.ndarray, dist) -> None:
    """One halo exchange of a per-atom FP64 array (local order, in place): the
    owned values peers hold as ghosts go out, this rank's ghosts come in."""
    import torch
    ws = dist.get_world_size()
    for q in range(ws):
        if q == p.rank:
            continue
        out = torch.as_tensor(values[p.send[q]]) if q in p.send else None
        inn = torch.zeros(len(p.recv[q]), dtype=torch.float64) if q in p.recv else None
        if p.rank < q:
            if out is not None and out.numel():
                dist.send(out, q)
            if inn is not None and inn.numel():
                dist.recv(inn, q)
        else:
            if inn is not None and inn.numel():
                dist.recv(inn, q)
            if out is not None and out.numel():
                dist.send(out, q)
        if inn is not None and inn.numel():
            values[p.recv[q]] = inn.numpy()
