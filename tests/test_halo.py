"""Halo logic of the domain-decomposed design (paper_1810_12357_gb300.halo) on
the CPU: the oracle's Jacobi substeps run rank by rank on slabs of one system,
with the ghost temperatures exchanged before every substep, must give every
atom the value of the undivided run bit for bit.  Three slabs in one process,
and two gloo ranks as separate processes (no GPU)."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import halo
from paper_1810_12357_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_SUB = 30


def _system():
    s = I.track_system(8, 3, peak=20000.0, r0=6.0)
    p = I.params_track()
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    sim.set_te(s.Te)
    sim.build(s.x, s.v)
    return s, p, sim


def _step(sim, p, rowptr, col, T, Tl, chi, A, n):
    st, _ = oracle.substeps(rowptr, col, T, Tl, chi, A, n, p["dt_sub"], p["Tmax"], sim.K, sim.cG, sim.VG)
    assert st == n


def _whole(s, p, sim):
    T, A = s.Te.copy(), np.zeros(s.n)
    _step(sim, p, sim.rowptr, sim.col, T, sim.Tl.copy(), sim.chi.copy(), A, N_SUB)
    return T, A


def test_three_slabs_in_one_process_equal_the_whole_system():
    s, p, sim = _system()
    T_ref, A_ref = _whole(s, p, sim)
    owner = halo.slab_owner(s.x, s.box, 3)
    plans = [halo.plan(sim.rowptr, sim.col, owner, r) for r in range(3)]
    halo.link_sends(plans)
    loc_T = [s.Te[pl.local_ids].copy() for pl in plans]
    loc_A = [np.zeros(pl.local_ids.size) for pl in plans]
    for pl in plans:
        assert pl.n_owned == int((owner == pl.rank).sum()) and len(pl.recv) > 0
    for _ in range(N_SUB):
        # exchange: every ghost takes its owner's current value
        for pl in plans:
            for q, idx in pl.send.items():
                dst = plans[q]
                loc_T[q][dst.recv[pl.rank]] = loc_T[pl.rank][idx]
        for r, pl in enumerate(plans):
            chi = np.where(pl.owned_mask, sim.chi[pl.local_ids], 0).astype(np.uint8)
            _step(sim, p, pl.rowptr, pl.col, loc_T[r], sim.Tl[pl.local_ids].copy(), chi, loc_A[r], 1)
    T = np.empty(s.n)
    A = np.empty(s.n)
    for r, pl in enumerate(plans):
        T[pl.local_ids[pl.owned_mask]] = loc_T[r][pl.owned_mask]
        A[pl.local_ids[pl.owned_mask]] = loc_A[r][pl.owned_mask]
    assert np.array_equal(T, T_ref)
    assert np.array_equal(A, A_ref)
    assert np.max(np.abs(T_ref - s.Te)) > 1.0


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    s, p, sim = _system()
    owner = halo.slab_owner(s.x, s.box, ws)
    pl = halo.plan(sim.rowptr, sim.col, owner, rank)
    halo.exchange_plan(pl, dist)
    T = s.Te[pl.local_ids].copy()
    A = np.zeros(pl.local_ids.size)
    chi = np.where(pl.owned_mask, sim.chi[pl.local_ids], 0).astype(np.uint8)
    for _ in range(N_SUB):
        halo.exchange_values(pl, T, dist)
        _step(sim, p, pl.rowptr, pl.col, T, sim.Tl[pl.local_ids].copy(), chi, A, 1)
    q.put((rank, pl.local_ids[pl.owned_mask], T[pl.owned_mask], A[pl.owned_mask]))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def test_two_gloo_ranks_equal_the_whole_system():
    s, p, sim = _system()
    T_ref, A_ref = _whole(s, p, sim)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    T = np.full(s.n, np.nan)
    A = np.full(s.n, np.nan)
    for rank, ids, Tr, Ar in res:
        T[ids] = Tr
        A[ids] = Ar
    assert np.array_equal(T, T_ref)
    assert np.array_equal(A, A_ref)


# ---- domains rebuilt every MD step from owned atoms and ghost positions ----

N_MD, N_SUB_MD = 3, 20


def _md_system(couple_mode=0):
    # a hot track on a lattice displaced by 0.1 A with 2,000 K velocities; the
    # slab faces of 2 and 3 domains (12 cells) lie on lattice planes, so atoms
    # cross them within the run
    s = I.track_system(12, 5, peak=20000.0, r0=6.0, disp_sigma=0.1, T_lat=2000.0)
    p = dict(I.params_track(), couple_mode=couple_mode, frozen=0, dt_sub=5e-3, kappa0=40.0,
             vatom=float(np.prod(s.box)) / s.n)
    return s, p


def oracle_domains(domains, exchange, allreduce, p, n_md, n_sub):
    """The oracle's MD steps on slab domains: the same sequence as
    halo.run_domains (migration, ghosts, build on the local positions, means of
    the owned atoms summed over the domains, ghost temperatures before every
    substep, hand-over with each atom's Langevin numbers keyed by its global id
    and the system's MD step, free flight); exchange / allreduce act on all of
    this process's domains at once."""
    import torch
    dt_md = n_sub * p["dt_sub"]
    t = 0.0
    for step in range(n_md):
        if step > 0:
            for d, i in zip(domains, exchange([d.migration_out() for d in domains])):
                d.migration_in(i)
        locs = [d.assemble(i) for d, i in zip(domains, exchange([d.ghosts_out() for d in domains]))]
        sims, sums = [], []
        for d, loc in zip(domains, locs):
            n = int(loc.ids.shape[0])
            sim = oracle.OracleSim(p, d.box, d.periodic, d.mass_amu, np.zeros(n, dtype=np.int32))
            sim.set_te(loc.T.numpy())
            sim.rng_ids, sim.md_step = loc.ids.numpy(), step
            x, v = loc.x.numpy().copy(), loc.v.numpy().copy()
            sim.build(x, v)
            k = loc.owned_idx.numpy()
            ke = 0.5 * sim.mass[k] * (v[k] * v[k]).sum(axis=1) * oracle.MVV_EV
            sums.append(torch.tensor([float(sim.T[k].sum()), float(ke.sum()), float(k.size)], dtype=torch.float64))
            sims.append((sim, x, v))
        for (sim, _, _), s in zip(sims, allreduce(sums)):
            N = float(s[2])
            sim.set_step_means(float(s[0]) / N, float(s[1]) / (1.5 * oracle.KB_EV * N))
        for kk in range(n_sub):
            outs = [{q: torch.as_tensor(sim.T[i.numpy()]) for q, i in loc.send.items()}
                    for (sim, _, _), loc in zip(sims, locs)]
            for (sim, _, _), loc, got in zip(sims, locs, exchange(outs)):
                for q, i in loc.recv.items():
                    sim.T[i.numpy()] = got[q].numpy()
            for sim, _, _ in sims:
                sim.substeps(1, t + kk * p["dt_sub"])
        for d, (sim, x, v), loc in zip(domains, sims, locs):
            sim.couple(v, dt_md)
            x = I.wrap(x + v * dt_md, np.asarray(d.box), np.asarray(d.periodic))
            d.take_owned(loc, torch.as_tensor(x), torch.as_tensor(v), torch.as_tensor(sim.T))
        t += dt_md


def _undivided(s, p):
    sys.path.insert(0, os.path.dirname(__file__))
    from _drive import run_oracle
    sim, x, v = run_oracle(s, p, N_MD, N_SUB_MD)
    return sim.T, x, v


def _collect(domains, n):
    T, x, v = np.full(n, np.nan), np.full((n, 3), np.nan), np.full((n, 3), np.nan)
    for d in domains:
        ids = d.ids.numpy()
        T[ids], x[ids], v[ids] = d.T.numpy(), d.x.numpy(), d.v.numpy()
    return T, x, v


def _compare(T, x, v, Tr, xr, vr):
    assert not np.isnan(T).any()
    assert float(np.max(np.abs(T - Tr) / Tr)) < 1e-12
    assert float(np.max(np.abs(v - vr))) < 1e-12 * float(np.abs(vr).max())
    assert float(np.max(np.abs(x - xr))) < 1e-12


@pytest.mark.parametrize("couple_mode", [0, 1])
def test_three_domains_rebuilt_every_md_step_equal_the_whole_system(couple_mode):
    # couple_mode 1: the Langevin hand-over, its numbers keyed by global ids
    s, p = _md_system(couple_mode)
    Tr, xr, vr = _undivided(s, p)
    reach = p["rc"] + 1e-5
    domains = [halo.SlabDomain.from_system(r, 3, s, reach) for r in range(3)]
    ids0 = [set(d.ids.tolist()) for d in domains]
    oracle_domains(domains, halo.LocalComm.exchange_all, halo.LocalComm.allreduce_all, p, N_MD, N_SUB_MD)
    # atoms crossed slab faces, and every atom is owned once
    moved = sum(len(set(d.ids.tolist()) - i0) for d, i0 in zip(domains, ids0))
    assert moved > 0
    assert sum(int(d.ids.shape[0]) for d in domains) == s.n
    _compare(*_collect(domains, s.n), Tr, xr, vr)


def _rank_md(rank, ws, port, q, couple_mode=0):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import test_halo as TH
    s, p = TH._md_system(couple_mode)
    comm = halo.DistComm(dist)
    d = halo.SlabDomain.from_system(rank, ws, s, p["rc"] + 1e-5)
    TH.oracle_domains([d], lambda outs: [comm.exchange(outs[0])], lambda ts: [comm.allreduce_sum(ts[0])], p,
                      TH.N_MD, TH.N_SUB_MD)
    q.put((d.ids.numpy(), d.T.numpy(), d.x.numpy(), d.v.numpy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("couple_mode", [0, 1])
def test_two_gloo_ranks_with_domains_rebuilt_every_md_step(couple_mode):
    s, p = _md_system(couple_mode)
    Tr, xr, vr = _undivided(s, p)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_md, args=(r, 2, port, q, couple_mode)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    T, x, v = np.full(s.n, np.nan), np.full((s.n, 3), np.nan), np.full((s.n, 3), np.nan)
    for ids, Tq, xq, vq in res:
        assert np.all(np.isnan(T[ids]))          # owned by one rank only
        T[ids], x[ids], v[ids] = Tq, xq, vq
    _compare(T, x, v, Tr, xr, vr)
