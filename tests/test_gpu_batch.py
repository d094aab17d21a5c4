"""Batched replicas (ehc_batch_*): one substep launch over the (replica, row)
work list of all replicas must give each replica exactly what a single context
gives it, and agree with the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I

from _drive import run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _concat(systems):
    x = np.concatenate([s.x for s in systems])
    v = np.concatenate([s.v for s in systems])
    Te = np.concatenate([s.Te for s in systems])
    return x, v, Te


def _run_batch(systems, p, n_md, n_sub):
    import torch
    from paper_1810_12357_gb300 import EhcBatch
    b = EhcBatch(p, systems)
    x, v, Te = _concat(systems)
    x = torch.as_tensor(x, device="cuda").contiguous()
    v = torch.as_tensor(v, device="cuda").contiguous()
    b.set_te(torch.as_tensor(Te, device="cuda"))
    dt_md = n_sub * p["dt_sub"]
    for step in range(n_md):
        b.build_neighbors(x, v)
        b.substep(n_sub, step * dt_md)
        b.couple(v, dt_md)
        b.drift(x, v, dt_md)
    torch.cuda.synchronize()
    return b, x, v


@pytest.mark.parametrize("couple_mode,skin", [(0, 0.0), (1, 0.0), (1, 0.3)])
def test_batch_equals_single_contexts(couple_mode, skin):
    # skin 0.3: the bench's batch configuration (each replica's list from its own
    # skin candidates)
    systems = I.batch_replicas(5, 41, n_min=1500, n_max=12000)
    p = dict(I.params_track(), couple_mode=couple_mode, Tmax=1e5, skin=skin)
    b, xb, vb = _run_batch(systems, p, 3, 40)
    Tb = b.get_te().cpu().numpy()
    vb = vb.cpu().numpy()
    for r, s in enumerate(systems):
        g, xg, vg = run_gpu(s, p, 3, 40)
        lo, hi = b.offsets[r], b.offsets[r] + s.n
        assert np.array_equal(Tb[lo:hi], g.get_te().cpu().numpy())
        assert np.array_equal(vb[lo:hi], vg.cpu().numpy())
        eb, eg = b.energy(r), g.energy()
        assert eb["E_e"] == eg["E_e"] and eb["E_lat"] == eg["E_lat"]


@pytest.mark.parametrize("skin", [0.0, 0.3])
def test_batch_replica_matches_oracle(skin):
    systems = I.batch_replicas(4, 42, n_min=2000, n_max=8000)
    p = dict(I.params_track(), skin=skin)
    b, _, _ = _run_batch(systems, p, 2, 50)
    Tb = b.get_te().cpu().numpy()
    for r, s in enumerate(systems):
        sim, _, _ = run_oracle(s, p, 2, 50)
        lo = b.offsets[r]
        err = float(np.max(np.abs(Tb[lo:lo + s.n] - sim.T) / sim.T))
        assert err < 1e-4, (r, err)
        assert abs(b.energy(r)["drift"]) < 1e-8


@pytest.mark.parametrize("batched", [False, True])
def test_tile_widths_and_tuner_give_identical_results(batched):
    # the 128- and 256-thread forms of the row-tile kernel, its persistent grid's
    # share of the resident CTAs, and the tuner's choice among them change only the
    # schedule: results are bit-identical
    systems = I.batch_replicas(4, 9, n_min=8000, n_max=40000)
    res = []
    for tt, q in ((256, 0), (128, 0), (256, 2), (128, 3), (0, 0)):
        p = dict(I.params_track(), tile_threads=tt, tile_grid_quarters=q)
        if batched:
            b, _, _ = _run_batch(systems, p, 2, 20)
            res.append(b.get_te().cpu().numpy())
            if tt == 0:
                assert b.tuning()[0] in (128, 256) and b.tuning()[1] in (2, 3, 4)
        else:
            g, _, _ = run_gpu(systems[0], p, 2, 20)
            res.append(g.get_te().cpu().numpy())
            if tt == 0:
                assert g.tuning()[0] in (128, 256) and g.tuning()[1] in (2, 3, 4)
    for r in res[1:]:
        assert np.array_equal(res[0], r)


def test_tuning_cache_keeps_the_choice(tmp_path, monkeypatch):
    # the tuner's choice is stored per GPU and shape and reused by the next context
    import json
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcBatch
    monkeypatch.setenv("EHC_TUNE_CACHE", str(tmp_path / "tuning.json"))
    s = I.track_system(16, 3, r0=10.0)
    p = I.params_track()
    x = torch.as_tensor(s.x, device="cuda")
    v = torch.as_tensor(s.v, device="cuda")
    g = Ehc(p, s, tune_cache=True)
    g.set_te(s.Te)
    g.build_neighbors(x, v)
    g.substep(20)
    choice = g.tuning()
    d = json.load(open(tmp_path / "tuning.json"))
    assert list(d.values())[0] and choice[0] in (128, 256)
    # a new context of the same shape starts with it (no tuning: a short call already shows it)
    h = Ehc(p, s, tune_cache=True)
    h.set_te(s.Te)
    h.build_neighbors(x, v)
    h.substep(2)
    assert h.tuning() == choice
    # the batch form
    systems = I.batch_replicas(3, 8, n_min=8000, n_max=30000)
    b, _, _ = _run_batch(systems, p, 1, 20)
    bb = EhcBatch(p, systems, tune_cache=True)
    bb.set_te(torch.as_tensor(np.concatenate([q.Te for q in systems]), device="cuda"))
    bb.build_neighbors(torch.as_tensor(np.concatenate([q.x for q in systems]), device="cuda").contiguous(),
                       torch.as_tensor(np.concatenate([q.v for q in systems]), device="cuda").contiguous())
    bb.substep(20)
    cb = bb.tuning()
    b2 = EhcBatch(p, systems, tune_cache=True)
    assert b2.params.get("tile_threads") == cb[0] and b2.params.get("tile_grid_quarters") == cb[1]


def test_fullsize_batch_sampled_replicas():
    """The batched workload at its full size (256 replicas, seed 4: about 33 M
    atoms) in one batch: one MD step of 20 substeps; three replicas (the smallest,
    a middle one and the largest) against the oracle run of the whole replica."""
    systems = I.batch_replicas(256, 4)
    p = I.params_track()
    sizes = np.array([s.n for s in systems])
    assert sizes.sum() > 30_000_000
    b, _, _ = _run_batch(systems, p, 1, 20)
    Tb = b.get_te().cpu().numpy()
    order = np.argsort(sizes)
    for r in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        s = systems[r]
        sim, _, _ = run_oracle(s, p, 1, 20)
        lo = b.offsets[r]
        err = float(np.max(np.abs(Tb[lo:lo + s.n] - sim.T) / sim.T))
        assert err < 1e-4, (r, s.n, err)
        assert abs(b.energy(r)["drift"]) < 1e-9
        print(f"full-size batch: replica {r} ({s.n:,} atoms) T_e err {err:.2e}")


def test_small_hot_replicas_keep_energy_over_50_md_steps():
    """The batch workload's smallest replicas with the hottest spots (8,788-atom
    cells, peaks of 20,000 K and more), 50 MD steps of 100 substeps in one batch:
    each replica's ledger drift stays within 1e-9.  The single-precision path's
    pair sums are compensated and its products added exactly, so the energy of a
    small hot system does not drift by each atom's rounding."""
    systems = I.batch_replicas(256, 4)
    pick = [r for r, s in enumerate(systems) if s.n < 10000 and s.Te.max() >= 20000.0][:4]
    assert len(pick) >= 2
    sel = [systems[r] for r in pick]
    b, _, _ = _run_batch(sel, I.params_track(), 50, 100)
    drifts = [b.energy(r)["drift"] for r in range(len(sel))]
    print("small hot replicas (" + ", ".join(f"{s.n} atoms, {s.Te.max():.0f} K" for s in sel) +
          "): drift after 50 MD steps " + ", ".join(f"{d:.1e}" for d in drifts))
    assert max(abs(d) for d in drifts) < 1e-9
