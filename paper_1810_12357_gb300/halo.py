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


# ---------------------------------------------------------------------------
# Domains rebuilt every MD step without the global neighbour list.
#
# A rank keeps only its owned atoms between MD steps (original id, position,
# velocity, electronic temperature).  At every neighbour rebuild:
#   1. atoms whose position left the slab migrate to their new owner;
#   2. every rank sends each peer its owned atoms within `reach` (the cutoff, with
#      a margin for the grid rounding) of the peer's slab, measured along the slab
#      axis: every neighbour of a peer's owned atom is among them;
#   3. the local system is the owned atoms and the received ghosts, ascending by
#      original id, so every owned atom's neighbour row keeps the global order.
# Then the context (or the oracle) of the rank builds its neighbour list from the
# local positions; ghost rows are incomplete, which does not matter because the
# ghosts' values are overwritten before every substep (exchange_ghosts).  The
# system means of the MD step are all-reduced from the owned atoms' sums.
# Messages are float64 tensors [k, 8] = (id, x, v, T); ids are exact in float64
# below 2^53.  The tensors may live on the GPU (NCCL moves them) or on the host.

class DistComm:
    """Exchanges between this rank and its peers over torch.distributed (NCCL
    for CUDA tensors, gloo for host tensors); the lower rank of a pair sends
    first, so no pair waits on itself."""

    def __init__(self, dist):
        self.dist = dist
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()

    def exchange(self, out: dict) -> dict:
        """out: peer -> tensor [k, w] (any k >= 0, same w and dtype for every
        pair); returns peer -> received tensor, for every peer."""
        import torch
        d = self.dist
        res = {}
        for q in range(self.size):
            if q == self.rank:
                continue
            t = out[q].contiguous()
            cnt = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
            got = torch.zeros(1, dtype=torch.int64, device=t.device)
            first = self.rank < q
            if first:
                d.send(cnt, q)
                d.recv(got, q)
            else:
                d.recv(got, q)
                d.send(cnt, q)
            r = torch.empty((int(got.item()),) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
            if first:
                if t.shape[0]:
                    d.send(t, q)
                if r.shape[0]:
                    d.recv(r, q)
            else:
                if r.shape[0]:
                    d.recv(r, q)
                if t.shape[0]:
                    d.send(t, q)
            res[q] = r
        return res

    def exchange_fixed(self, out: dict, sizes: dict) -> dict:
        """As exchange, with the receive sizes known (the per-substep ghost values)."""
        import torch
        d = self.dist
        res = {}
        for q in range(self.size):
            if q == self.rank:
                continue
            t = out[q].contiguous()
            r = torch.empty(sizes[q], dtype=t.dtype, device=t.device)
            if self.rank < q:
                if t.numel():
                    d.send(t, q)
                if r.numel():
                    d.recv(r, q)
            else:
                if r.numel():
                    d.recv(r, q)
                if t.numel():
                    d.send(t, q)
            res[q] = r
        return res

    def allreduce_sum(self, t):
        self.dist.all_reduce(t)
        return t


class LocalComm:
    """Several domains stepped together in one process (one context per domain
    on one device, or oracle domains): the same exchanges as DistComm, done by
    the caller for all domains at once (exchange_all)."""

    def __init__(self, size: int):
        self.size = size

    @staticmethod
    def exchange_all(outs: list) -> list:
        """outs[r]: peer -> tensor from domain r; returns, for every domain, peer ->
        what that peer sent it."""
        return [{q: outs[q][r] for q in range(len(outs)) if q != r} for r in range(len(outs))]

    @staticmethod
    def allreduce_all(ts: list):
        tot = ts[0].clone()
        for t in ts[1:]:
            tot += t
        return [tot.clone() for _ in ts]


@dataclass
class LocalSystem:
    """One rank's local system of an MD step (ascending original ids)."""
    ids: "object"          # int64 [n_local]
    x: "object"            # [n_local, 3]
    v: "object"            # [n_local, 3]
    T: "object"            # [n_local]
    owned: "object"        # bool [n_local]
    owned_idx: "object"    # int64 local indices of the owned atoms
    send: dict             # peer -> int64 local indices of owned atoms the peer holds as ghosts
    recv: dict             # peer -> int64 local indices of ghosts owned by the peer (its send order)


class SlabDomain:
    """The owned atoms of one rank: equal slabs of the box along `axis`."""

    def __init__(self, rank: int, n_ranks: int, box, periodic, reach: float, ids, x, v, T, axis: int = 0,
                 mass_amu=(63.546,)):
        import torch
        self.rank, self.n_ranks, self.axis = rank, n_ranks, axis
        self.mass_amu = np.asarray(mass_amu, dtype=np.float64)
        self.box = [float(b) for b in box]
        self.periodic = [int(p) for p in periodic]
        self.reach = float(reach)
        self.ids = torch.as_tensor(ids, dtype=torch.int64)
        dev = self.ids.device
        self.x = torch.as_tensor(x, dtype=torch.float64, device=dev)
        self.v = torch.as_tensor(v, dtype=torch.float64, device=dev)
        self.T = torch.as_tensor(T, dtype=torch.float64, device=dev)

    @classmethod
    def from_system(cls, rank, n_ranks, system, reach, device="cpu", axis: int = 0):
        import torch
        own = slab_owner(system.x, system.box, n_ranks, axis) == rank
        ids = np.flatnonzero(own)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=device)
        if np.asarray(system.mass_amu).shape[0] != 1:
            raise ValueError("slab domains carry one atom type")
        return cls(rank, n_ranks, system.box, system.periodic, reach, t(ids), t(system.x[ids]), t(system.v[ids]),
                   t(system.Te[ids]), axis, system.mass_amu)

    # ---- geometry ----
    def _slab(self, r: int):
        L = self.box[self.axis]
        return r * L / self.n_ranks, (r + 1) * L / self.n_ranks

    def owner_of(self, x):
        import torch
        L = self.box[self.axis]
        r = torch.floor(x[:, self.axis] / L * self.n_ranks).to(torch.int64)
        return r.clamp(0, self.n_ranks - 1)

    def _near(self, x, r: int):
        """Atoms within reach of slab r along the axis (periodic wrap if periodic)."""
        import torch
        lo, hi = self._slab(r)
        u = x[:, self.axis]
        below = lo - u
        above = u - hi
        if self.periodic[self.axis]:
            L = self.box[self.axis]
            below = torch.remainder(below, L)
            above = torch.remainder(above, L)
        inside = (u >= lo) & (u < hi)
        return inside | (below <= self.reach) | (above <= self.reach)

    # ---- per-MD-step steps ----
    def _pack(self, sel):
        import torch
        return torch.cat([self.ids[sel].to(torch.float64)[:, None], self.x[sel], self.v[sel], self.T[sel][:, None]],
                         dim=1)

    def migration_out(self) -> dict:
        """Peer -> rows (id, x, v, T) of the owned atoms that now belong to it;
        those atoms leave this domain."""
        own = self.owner_of(self.x)
        out = {q: self._pack(own == q) for q in range(self.n_ranks) if q != self.rank}
        keep = own == self.rank
        self.ids, self.x, self.v, self.T = self.ids[keep], self.x[keep], self.v[keep], self.T[keep]
        return out

    def migration_in(self, got: dict) -> None:
        import torch
        rows = [g for g in got.values() if g.shape[0]]
        if rows:
            r = torch.cat(rows)
            self.ids = torch.cat([self.ids, r[:, 0].to(torch.int64)])
            self.x = torch.cat([self.x, r[:, 1:4]])
            self.v = torch.cat([self.v, r[:, 4:7]])
            self.T = torch.cat([self.T, r[:, 7]])
        o = torch.argsort(self.ids)
        self.ids, self.x, self.v, self.T = self.ids[o], self.x[o], self.v[o], self.T[o]

    def ghosts_out(self) -> dict:
        """Peer -> rows of the owned atoms (ascending id) within reach of its slab."""
        self._ghost_sel = {q: self._near(self.x, q) for q in range(self.n_ranks) if q != self.rank}
        return {q: self._pack(sel) for q, sel in self._ghost_sel.items()}

    def assemble(self, got: dict) -> LocalSystem:
        """The local system from the owned atoms and the received ghosts."""
        import torch
        parts = [self._pack(torch.ones_like(self.ids, dtype=torch.bool))]
        src = [torch.full((self.ids.shape[0],), self.rank, dtype=torch.int64, device=self.ids.device)]
        for q in sorted(got):
            parts.append(got[q])
            src.append(torch.full((got[q].shape[0],), q, dtype=torch.int64, device=self.ids.device))
        rows = torch.cat(parts)
        src = torch.cat(src)
        ids = rows[:, 0].to(torch.int64)
        o = torch.argsort(ids)
        rows, src, ids = rows[o], src[o], ids[o]
        owned = src == self.rank
        pos = torch.arange(ids.shape[0], device=ids.device)
        # what each peer holds of ours: our owned atoms it received, ascending id,
        # which are our owned rows in the same order
        own_pos = pos[owned]
        send = {q: own_pos[sel] for q, sel in self._ghost_sel.items()}
        recv = {q: pos[src == q] for q in got}
        return LocalSystem(ids=ids, x=rows[:, 1:4].contiguous(), v=rows[:, 4:7].contiguous(),
                           T=rows[:, 7].contiguous(), owned=owned, owned_idx=own_pos, send=send, recv=recv)

    def take_owned(self, loc: LocalSystem, x, v, T) -> None:
        """Carry the owned atoms' state of the finished MD step (local arrays)."""
        k = loc.owned_idx
        self.ids, self.x, self.v, self.T = loc.ids[k], x[k].clone(), v[k].clone(), T[k].clone()


def run_domains(domains: list, comm, params: dict, n_md: int, n_sub: int, t0: float = 0.0, md_step0: int = 0):
    """Advance the domains of this process by n_md MD steps of the whole path on
    the CUDA library, one context per domain and MD step: migration, ghosts,
    neighbour build from the local positions, the system means all-reduced from
    the owned atoms' sums (ehc_sums_at, ehc_set_step_means), before every substep
    the ghost temperatures packed on the device (ehc_get_te_at), exchanged and
    unpacked (ehc_set_te_at), then the hand-over and the drift.  comm: DistComm
    (one domain per process, tensors on this rank's GPU) or LocalComm (all
    domains of the system in this process).  params must fix vatom (the system's
    volume per atom): a domain's own volume per atom is not the system's.  The
    Langevin hand-over draws each atom's numbers by its global id and the system's
    MD step (md_step0 + the step of this call; ehc_set_rng_ids), as the undivided
    run does."""
    import torch
    from . import Ehc
    if not params.get("vatom"):
        raise ValueError("params['vatom'] must be the whole system's volume per atom")
    local = isinstance(comm, LocalComm)

    def xchg(outs):
        return LocalComm.exchange_all(outs) if local else [comm.exchange(outs[0])]

    def xchg_fixed(outs, sizes):
        return LocalComm.exchange_all(outs) if local else [comm.exchange_fixed(outs[0], sizes[0])]

    def allred(ts):
        return LocalComm.allreduce_all(ts) if local else [comm.allreduce_sum(ts[0])]

    dt_md = n_sub * params["dt_sub"]
    kb = 8.617333262e-5
    t = t0
    for step in range(n_md):
        if step > 0:
            ins = xchg([d.migration_out() for d in domains])
            for d, i in zip(domains, ins):
                d.migration_in(i)
        ins = xchg([d.ghosts_out() for d in domains])
        locs = [d.assemble(i) for d, i in zip(domains, ins)]
        ctxs, sums = [], []
        for d, loc in zip(domains, locs):
            n = int(loc.ids.shape[0])
            g = Ehc(params, n=n, box=d.box, periodic=d.periodic, mass_amu=d.mass_amu,
                    types=np.zeros(n, dtype=np.int32))
            g.set_te(loc.T)
            g.set_rng_ids(loc.ids, md_step0 + step)
            g.build_neighbors(loc.x, loc.v)
            st, ke = g.sums_at(loc.owned_idx.to(torch.int32))
            sums.append(torch.tensor([st, ke, float(loc.owned_idx.shape[0])], dtype=torch.float64,
                                     device=loc.ids.device))
            ctxs.append(g)
        tot = allred(sums)
        for g, s in zip(ctxs, tot):
            s = s.cpu()
            N = float(s[2])
            g.set_step_means(float(s[0]) / N, float(s[1]) / (1.5 * kb * N))
        send_idx = [{q: i.to(torch.int32) for q, i in loc.send.items()} for loc in locs]
        recv_idx = [{q: i.to(torch.int32) for q, i in loc.recv.items()} for loc in locs]
        sizes = [{q: int(i.shape[0]) for q, i in loc.recv.items()} for loc in locs]
        for k in range(n_sub):
            outs = [{q: g.get_te_at(i) for q, i in si.items()} for g, si in zip(ctxs, send_idx)]
            got = xchg_fixed(outs, sizes)
            for g, ri, gi in zip(ctxs, recv_idx, got):
                for q, idx in ri.items():
                    if idx.numel():
                        g.set_te_at(idx, gi[q])
            for g in ctxs:
                g.substep(1, t + k * params["dt_sub"])
        for d, g, loc in zip(domains, ctxs, locs):
            x, v = loc.x.clone(), loc.v.clone()
            g.couple(v, dt_md)
            g.drift(x, v, dt_md)
            d.take_owned(loc, x, v, g.get_te())
            g.close()
        t += dt_md
