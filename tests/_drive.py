"""Run the same MD-step sequence through the CUDA library and through the CPU
oracle, from the same seeded inputs (test infrastructure)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1810_12357_gb300 import inputs as I


def run_oracle(system: I.System, p: dict, n_md: int, n_sub: int, dt_md: float | None = None,
               drift: bool = True, t0: float = 0.0, border=None):
    """The electrons and the lattice advance the same time per MD step unless
    dt_md is given: dt_md = n_sub * dt_sub.  border: per-atom fixed T_e (NaN: free)."""
    dt_md = n_sub * p["dt_sub"] if dt_md is None else dt_md
    sim = oracle.OracleSim(p, system.box, system.periodic, system.mass_amu, system.type, depth=system.depth)
    sim.set_te(system.Te)
    if border is not None:
        sim.set_border(border)
    x = system.x.copy()
    v = system.v.copy()
    t = t0
    for step in range(n_md):
        sim.build(x, v)
        sim.substeps(n_sub, t)
        t += n_sub * p["dt_sub"]
        sim.couple(v, dt_md)
        if drift and not p["frozen"]:
            x = I.wrap(x + v * dt_md, system.box, system.periodic)
    return sim, x, v


def run_gpu(system: I.System, p: dict, n_md: int, n_sub: int, dt_md: float | None = None,
            drift: bool = True, t0: float = 0.0, border=None):
    dt_md = n_sub * p["dt_sub"] if dt_md is None else dt_md
    import torch
    from paper_1810_12357_gb300 import Ehc
    g = Ehc(p, system)
    g.set_te(system.Te)
    if border is not None:
        g.set_border(border)
    if system.depth is not None:
        g.set_depth(system.depth)
    x = torch.as_tensor(system.x, device="cuda").contiguous()
    v = torch.as_tensor(system.v, device="cuda").contiguous()
    t = t0
    for step in range(n_md):
        g.build_neighbors(x, v)
        g.substep(n_sub, t)
        t += n_sub * p["dt_sub"]
        g.couple(v, dt_md)
        if drift and not p["frozen"]:
            g.drift(x, v, dt_md)
    torch.cuda.synchronize()
    return g, x, v
