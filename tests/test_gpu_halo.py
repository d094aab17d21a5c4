"""Device side of the domain-decomposed design on one GPU: one context per slab
(its owned atoms and the ghosts their rows reach, in the full periodic box),
the step means of the undivided system set on every domain (ehc_set_step_means),
and before every substep the ghost temperatures copied from their owners'
contexts (ehc_get_te_at / ehc_set_te_at, host-ordered: no kernel waits on
another).  The FP64 path gives every owned atom bit for bit the undivided
context's T_e (the same neighbour order, the same coefficients); the
single-precision row tiles agree to their truncation bound."""
import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import halo
from paper_1810_12357_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N_SUB = 20


def _domains(s, p, n_dom):
    import torch
    from paper_1810_12357_gb300 import Ehc
    rowptr, col = oracle.neighbors(s.x, s.box, s.periodic, p["rc"])
    owner = halo.slab_owner(s.x, s.box, n_dom)
    plans = [halo.plan(rowptr, col, owner, r) for r in range(n_dom)]
    halo.link_sends(plans)
    ctxs = []
    for pl in plans:
        ids = pl.local_ids
        sub = I.System(x=s.x[ids], v=s.v[ids], Te=s.Te[ids], box=s.box, periodic=s.periodic,
                       mass_amu=s.mass_amu, type=s.type[ids], a=s.a, name=f"domain_{pl.rank}")
        g = Ehc(p, sub)
        g.set_te(sub.Te)
        g.build_neighbors(torch.as_tensor(sub.x, device="cuda"), torch.as_tensor(sub.v, device="cuda"))
        ctxs.append(g)
    return plans, ctxs


KB_EV = 8.617333262e-5


def _run(s, p, n_dom, means="undivided"):
    import torch
    from paper_1810_12357_gb300 import Ehc
    ref = Ehc(p, s)
    ref.set_te(s.Te)
    ref.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    e = ref.energy()
    plans, ctxs = _domains(s, p, n_dom)
    if means == "undivided":
        Te_mean, Tlat = e["Te_mean_step"], e["Tlat_step"]
    else:
        # the all-reduce of a multi-GPU run: every domain's sums over its owned atoms
        sT = sK = 0.0
        for pl, g in zip(plans, ctxs):
            own = torch.as_tensor(np.flatnonzero(pl.owned_mask).astype(np.int32), device="cuda")
            a, b = g.sums_at(own)
            sT += a
            sK += b
        Te_mean, Tlat = sT / s.n, sK / (1.5 * KB_EV * s.n)
        assert Te_mean == pytest.approx(e["Te_mean_step"], rel=1e-13)
        assert Tlat == pytest.approx(e["Tlat_step"], rel=1e-13)
    for g in ctxs:
        g.set_step_means(Te_mean, Tlat)
        if means == "undivided":
            assert g.energy()["K_per_fs"] == e["K_per_fs"]
    sends = {(pl.rank, q): torch.as_tensor(idx.astype(np.int32), device="cuda")
             for pl in plans for q, idx in pl.send.items()}
    recvs = {(q, pl.rank): torch.as_tensor(idx.astype(np.int32), device="cuda")
             for pl in plans for q, idx in pl.recv.items()}
    for k in range(N_SUB):
        for (r, q), idx in sends.items():
            ctxs[q].set_te_at(recvs[(r, q)], ctxs[r].get_te_at(idx))
        for g in ctxs:
            g.substep(1, k * p["dt_sub"])
    ref.substep(N_SUB)
    T_ref = ref.get_te().cpu().numpy()
    T = np.full(s.n, np.nan)
    for pl, g in zip(plans, ctxs):
        Tl = g.get_te().cpu().numpy()
        T[pl.local_ids[pl.owned_mask]] = Tl[pl.owned_mask]
        assert g.energy()["device_error"] == 0
    return T, T_ref


def test_fp64_domains_equal_the_undivided_context():
    s = I.track_system(10, 3, peak=20000.0, r0=6.0)
    p = dict(I.params_track(), flux_prec=1)
    T, T_ref = _run(s, p, 2)
    assert np.array_equal(T, T_ref)
    assert np.max(np.abs(T_ref - s.Te)) > 1.0


def test_single_precision_domains_agree_with_the_undivided_context():
    s = I.track_system(12, 4, peak=20000.0, r0=6.0)
    p = I.params_track()
    T, T_ref = _run(s, p, 3)
    err = float(np.max(np.abs(T - T_ref) / T_ref))
    # the row tiles' series order differs at the domain edges (ghost rows) and after
    # each overwrite: truncation below 3e-8 of the pair term
    assert err < 1e-6, err
    print(f"single-precision domains vs undivided: {err:.1e}")


def test_domain_means_from_owned_sums():
    """The step means from each domain's sums over its owned atoms (ehc_sums_at),
    added over the domains as an all-reduce would: the FP64 domains agree with the
    undivided context to the rounding of the sums' order."""
    s = I.track_system(10, 3, peak=20000.0, r0=6.0)
    p = dict(I.params_track(), flux_prec=1)
    T, T_ref = _run(s, p, 2, means="sums")
    err = float(np.max(np.abs(T - T_ref) / T_ref))
    assert err < 1e-12, err


@pytest.mark.parametrize("flux_prec,couple_mode", [(1, 0), (0, 0), (1, 1)])
def test_domains_rebuilt_every_md_step_on_one_gpu(flux_prec, couple_mode):
    """halo.run_domains on one GPU: 2 and 3 slab domains of a system, each MD step
    rebuilt from its owned atoms and the ghosts within r_c of its slab (no global
    neighbour list), atoms migrating between domains, the means all-reduced from
    the owned atoms' sums, the ghost temperatures packed and unpacked on the device
    before every substep; against the undivided context.  FP64 flux: T_e within
    1e-11, positions and velocities 1e-12 (the all-reduced means differ from the
    undivided sums in the last bits); single-precision flux: T_e within 1e-7 (an
    overwritten ghost makes the next substep take the full series, where the
    undivided run takes each tile's own order).  couple_mode 1: the Langevin
    hand-over, each domain atom's numbers keyed by its global id and the system's
    MD step (ehc_set_rng_ids), as the undivided context draws them."""
    import torch
    import test_halo as TH
    from paper_1810_12357_gb300 import halo
    from _drive import run_gpu
    s, p = TH._md_system(couple_mode)
    p = dict(p, flux_prec=flux_prec)
    tol = 1e-11 if flux_prec == 1 else 1e-7
    g, xg, vg = run_gpu(s, p, TH.N_MD, TH.N_SUB_MD)
    Tr, xr, vr = g.get_te().cpu().numpy(), xg.cpu().numpy(), vg.cpu().numpy()
    for nd in (2, 3):
        domains = [halo.SlabDomain.from_system(r, nd, s, p["rc"] + 1e-5, device="cuda") for r in range(nd)]
        ids0 = [set(d.ids.tolist()) for d in domains]
        halo.run_domains(domains, halo.LocalComm(nd), p, TH.N_MD, TH.N_SUB_MD)
        assert sum(len(set(d.ids.tolist()) - i0) for d, i0 in zip(domains, ids0)) > 0
        T, x, v = np.full(s.n, np.nan), np.full((s.n, 3), np.nan), np.full((s.n, 3), np.nan)
        for d in domains:
            ids = d.ids.cpu().numpy()
            assert np.all(np.isnan(T[ids]))
            T[ids], x[ids], v[ids] = d.T.cpu().numpy(), d.x.cpu().numpy(), d.v.cpu().numpy()
        err = float(np.max(np.abs(T - Tr) / Tr))
        print(f"{nd} domains rebuilt every MD step (flux_prec {flux_prec}, couple_mode {couple_mode}): "
              f"T_e max rel err {err:.2e}, "
              f"x {np.max(np.abs(x - xr)):.1e} A, v {np.max(np.abs(v - vr)):.1e} A/fs")
        assert err < tol
        assert float(np.max(np.abs(x - xr))) < 1e3 * tol
        assert float(np.max(np.abs(v - vr))) < tol * float(np.abs(vr).max())


def test_rng_ids_key_the_langevin_stream():
    """ehc_set_rng_ids: ids equal to the caller index reproduce the default
    Langevin hand-over bit for bit; other ids or another MD step draw other
    numbers; the oracle keyed by the same ids agrees (velocities within 1e-6 of
    the largest: the GPU's Box-Muller runs in single precision); null ids return
    to the index."""
    import torch
    from paper_1810_12357_gb300 import Ehc
    s = I.track_system(6, 3, r0=5.0)
    p = dict(I.params_track(), couple_mode=1)
    n_sub, dt_md = 10, 10 * p["dt_sub"]
    ids_shift = np.arange(s.n, dtype=np.int64)[::-1].copy() + 1000

    def hand_over(ids, md_step):
        g = Ehc(p, s)
        g.set_te(s.Te)
        if ids is not False:
            g.set_rng_ids(None if ids is None else torch.as_tensor(ids, device="cuda"), md_step)
        x = torch.as_tensor(s.x, device="cuda").contiguous()
        v = torch.as_tensor(s.v, device="cuda").contiguous()
        g.build_neighbors(x, v)
        g.substep(n_sub, 0.0)
        g.couple(v, dt_md)
        torch.cuda.synchronize()
        return v.cpu().numpy()

    v_def = hand_over(False, 0)
    assert np.array_equal(hand_over(np.arange(s.n, dtype=np.int64), 0), v_def)
    assert np.array_equal(hand_over(None, 0), v_def)
    v_ids = hand_over(ids_shift, 0)
    v_step = hand_over(None, 3)
    assert not np.array_equal(v_ids, v_def) and not np.array_equal(v_step, v_def)
    # the oracle with the same ids and step
    for ids, step, vg in ((ids_shift, 0, v_ids), (None, 3, v_step)):
        sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
        sim.set_te(s.Te)
        sim.rng_ids, sim.md_step = ids, step
        x, v = s.x.copy(), s.v.copy()
        sim.build(x, v)
        sim.substeps(n_sub, 0.0)
        sim.couple(v, dt_md)
        assert float(np.max(np.abs(v - vg))) < 1e-6 * float(np.abs(v).max())
