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
