"""CPU oracle for the l2T-MD electronic heat-conduction step (arXiv 1810.12357).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is a plain FP64
restatement of the paper's equations (C loops in ``ehc_oracle.c`` plus the
bookkeeping below in numpy) and shares no code with the CUDA library.

Pins (tests/test_oracle_*.py) tie each function to something other than
itself: brute-force neighbour search, the perfect-FCC neighbour count, flux
antisymmetry and the uniform fixed point (Eq. HeatTransport), the Fourier-law
decay rate implied by Eq. Kij, exact electron/lattice energy balance
(Eqs. RateExchange, WorkDone, Xi), the two-bath equilibrium of the 1-D bar
(Sec. 3.1), and published Philox4x32-10 known-answer vectors.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

# CODATA 2018
KB_EV = 8.617333262e-5
KB_J = 1.380649e-23
EV_J = 1.602176634e-19
AMU_KG = 1.66053906660e-27
MVV_EV = AMU_KG * 1.0e10 / EV_J

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        u64 = ctypes.c_uint64
        L.oracle_quantize.argtypes = [i64, P, P, P, P, P]
        L.oracle_quantize.restype = ctypes.c_int
        for f in (L.oracle_neighbors_brute, L.oracle_neighbors_cells):
            f.argtypes = [i64, P, P, P, i64, P, P, i64]
            f.restype = i64
        L.oracle_lattice_temperature.argtypes = [i64, P, P, P, P, ctypes.c_int, P, P]
        L.oracle_lattice_temperature.restype = None
        L.oracle_pair_flux.argtypes = [dbl, dbl]
        L.oracle_pair_flux.restype = dbl
        L.oracle_flux_sum.argtypes = [i64, P, P, P, P]
        L.oracle_flux_sum.restype = None
        L.oracle_pair_dflux_a.argtypes = [dbl, dbl]
        L.oracle_pair_dflux_a.restype = dbl
        L.oracle_flux_vjp.argtypes = [i64, P, P, P, P, P]
        L.oracle_flux_vjp.restype = None
        L.oracle_substeps.argtypes = [i64, P, P, P, P, P, P, ctypes.c_int, dbl, dbl, dbl, dbl,
                                      dbl, P, P, dbl, dbl, dbl, P, P, P, P]
        L.oracle_substeps_local.argtypes = [i64, P, P, P, P, P, P, ctypes.c_int, dbl, dbl, dbl,
                                            ctypes.c_int, dbl, ctypes.c_int, dbl, dbl, dbl, dbl, dbl,
                                            P, P, dbl, P, P, P, P]
        L.oracle_substeps_local.restype = ctypes.c_int
        L.oracle_ce_energy.argtypes = [dbl, dbl, dbl]
        L.oracle_ce_energy.restype = dbl
        L.oracle_ce_energy_inv.argtypes = [dbl, dbl, dbl]
        L.oracle_ce_energy_inv.restype = dbl
        L.oracle_forces.argtypes = [i64, P, P, P, P, P, dbl, dbl, dbl, dbl, P, P]
        L.oracle_forces.restype = None
        L.oracle_morse.argtypes = [dbl, dbl, dbl, dbl, P, P]
        L.oracle_morse.restype = None
        L.oracle_kick.argtypes = [i64, P, P, P, dbl]
        L.oracle_kick.restype = None
        L.oracle_pair_weights.argtypes = [i64, P, P, P, P, P, dbl, i32, P]
        L.oracle_pair_weights.restype = None
        L.oracle_substeps.restype = ctypes.c_int
        L.oracle_philox4x32_10.argtypes = [P, P, P]
        L.oracle_philox4x32_10.restype = None
        L.oracle_gauss3.argtypes = [u64, u64, u64, P]
        L.oracle_gauss3.restype = None
        L.oracle_couple.argtypes = [i64, P, P, P, P, P, ctypes.c_int, ctypes.c_int, u64, u64,
                                    dbl, dbl, dbl, P, dbl, dbl, P]
        L.oracle_couple.restype = i64
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


# --------------------------------------------------------------------------
# neighbour lists (Sec. 2: j with |x_j - x_i| <= r_c)

def quantize(x: np.ndarray, box, periodic):
    x = np.ascontiguousarray(x, dtype=np.float64)
    box = np.ascontiguousarray(box, dtype=np.float64)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    q = np.empty((x.shape[0], 3), dtype=np.int32)
    Lq = np.empty(3, dtype=np.int64)
    rc = lib().oracle_quantize(x.shape[0], _p(x), _p(box), _p(per), _p(q), _p(Lq))
    if rc != 0:
        raise ValueError(f"oracle_quantize failed ({rc})")
    return q, Lq


def rc_fixed(rc_A: float) -> int:
    return int(np.rint(rc_A * 1048576.0))


def neighbors(x: np.ndarray, box, periodic, rc_A: float, method: str = "cells",
              cap_per_atom: int = 64):
    """Full neighbour list in original ids: (rowptr int64 [N+1], col int32)."""
    q, Lq = quantize(x, box, periodic)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    n = q.shape[0]
    cap = max(1, n * cap_per_atom)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(cap, dtype=np.int32)
    f = lib().oracle_neighbors_brute if method == "brute" else lib().oracle_neighbors_cells
    nnz = f(n, _p(q), _p(Lq), _p(per), rc_fixed(rc_A), _p(rowptr), _p(col), cap)
    if nnz < 0:
        raise ValueError(f"neighbour list capacity exceeded ({nnz})")
    return rowptr, col[:nnz].copy()


# --------------------------------------------------------------------------
# local lattice temperature (Sec. 2)

def lattice_temperature(rowptr, col, v, mass_of_atom, dof_mode: int = 0):
    n = rowptr.shape[0] - 1
    v = np.ascontiguousarray(v, dtype=np.float64)
    m = np.ascontiguousarray(mass_of_atom, dtype=np.float64)
    Tl = np.empty(n)
    Ks = np.empty(n)
    lib().oracle_lattice_temperature(n, _p(rowptr), _p(col), _p(v), _p(m), int(dof_mode),
                                     _p(Tl), _p(Ks))
    return Tl, Ks


def pair_flux(a: float, b: float) -> float:
    return float(lib().oracle_pair_flux(float(a), float(b)))


def flux_sum(rowptr, col, theta):
    """F_i = sum_j f(theta_i, theta_j) over the list (Eq. HeatTransport, flux part)."""
    n = rowptr.shape[0] - 1
    th = np.ascontiguousarray(theta, dtype=np.float64)
    F = np.empty(n)
    lib().oracle_flux_sum(n, _p(np.ascontiguousarray(rowptr, dtype=np.int64)),
                          _p(np.ascontiguousarray(col, dtype=np.int32)), _p(th), _p(F))
    return F


def pair_dflux_a(a: float, b: float) -> float:
    """d f(a, b) / d a of the pair term (Eq. HeatTransport)."""
    return lib().oracle_pair_dflux_a(float(a), float(b))


def flux_vjp(rowptr, col, theta, lam):
    """out_m = sum_i lam_i dF_i/dtheta_m: the transposed Jacobian of flux_sum."""
    n = rowptr.shape[0] - 1
    th = np.ascontiguousarray(theta, dtype=np.float64)
    lm = np.ascontiguousarray(lam, dtype=np.float64)
    out = np.empty(n)
    lib().oracle_flux_vjp(n, _p(np.ascontiguousarray(rowptr, dtype=np.int64)),
                          _p(np.ascontiguousarray(col, dtype=np.int32)), _p(th), _p(lm), _p(out))
    return out


def pair_weights(x, box, periodic, rowptr, col, S2_A2: float, n_shell: int):
    """Distance weights S2 / (n_shell r_ij^2) of the list entries (oracle_pair_weights)."""
    q, Lq = quantize(x, box, periodic)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    w = np.empty(col.shape[0])
    lib().oracle_pair_weights(rowptr.shape[0] - 1, _p(np.ascontiguousarray(rowptr, dtype=np.int64)),
                              _p(np.ascontiguousarray(col, dtype=np.int32)), _p(q), _p(Lq), _p(per),
                              float(S2_A2), int(n_shell), _p(w))
    return w


def substeps(rowptr, col, T, Tl, chi, A, n_sub, dt, Tmax, K, cG, VG, *, depth=None,
             source=None, Ce_SI=1.0, vatom_A3=1.0, t_start=0.0, Tfix=None, eres=None, weights=None):
    """In place on T and A; returns (status, E_src increment).  Tfix: per-atom
    border temperature (NaN: free atom); the kelvin sum the border absorbed is
    added to eres[0] (a one-element float64 array) when given."""
    n = rowptr.shape[0] - 1
    esrc = np.zeros(1)
    src = None
    if source is not None:
        src = np.ascontiguousarray([1.0, source["fluence_Jm2"], source["lp_A"], source["t0_fs"],
                                    source["sigma_fs"]], dtype=np.float64)
        depth = np.ascontiguousarray(depth, dtype=np.float64)
    if Tfix is not None:
        Tfix = np.ascontiguousarray(Tfix, dtype=np.float64)
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.float64)
    st = lib().oracle_substeps(n, _p(rowptr), _p(col), _p(T), _p(Tl), _p(chi), _p(A), int(n_sub),
                               float(dt), float(Tmax), float(K), float(cG), float(VG),
                               _p(depth) if depth is not None else None,
                               _p(src) if src is not None else None, float(Ce_SI),
                               float(vatom_A3), float(t_start), _p(esrc),
                               _p(Tfix) if Tfix is not None else None,
                               _p(eres) if eres is not None else None,
                               _p(weights) if weights is not None else None)
    return st, float(esrc[0])


def substeps_local(rowptr, col, T, Tl, chi, A, n_sub, dt, Tmax, *, kappa0, kappa_mode, Tlat, dim_d,
                   S2_A2, gamma, cap_SI, G, vatom_A3, depth=None, source=None, t_start=0.0, Tfix=None,
                   weights=None):
    """LOCAL per-atom C_e / kappa_e form (oracle_substeps_local), in place on T and
    A; returns (status, E_src increment [eV], border energy increment [eV])."""
    n = rowptr.shape[0] - 1
    esrc = np.zeros(1)
    eres = np.zeros(1)
    src = None
    if source is not None:
        src = np.ascontiguousarray([1.0, source["fluence_Jm2"], source["lp_A"], source["t0_fs"],
                                    source["sigma_fs"]], dtype=np.float64)
        depth = np.ascontiguousarray(depth, dtype=np.float64)
    if Tfix is not None:
        Tfix = np.ascontiguousarray(Tfix, dtype=np.float64)
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.float64)
    st = lib().oracle_substeps_local(n, _p(rowptr), _p(col), _p(T), _p(Tl), _p(chi), _p(A), int(n_sub),
                                     float(dt), float(Tmax), float(kappa0), int(kappa_mode), float(Tlat),
                                     int(dim_d), float(S2_A2), float(gamma), float(cap_SI), float(G),
                                     float(vatom_A3), _p(depth) if depth is not None else None,
                                     _p(src) if src is not None else None, float(t_start), _p(esrc),
                                     _p(Tfix) if Tfix is not None else None, _p(eres),
                                     _p(weights) if weights is not None else None)
    return st, float(esrc[0]), float(eres[0])


def ce_energy(T: float, gamma: float, cap: float) -> float:
    """U(T) = int_0^T min(gamma T', cap) dT' [J m^-3] (the C routine)."""
    return lib().oracle_ce_energy(float(T), float(gamma), float(cap))


def ce_energy_inv(U: float, gamma: float, cap: float) -> float:
    return lib().oracle_ce_energy_inv(float(U), float(gamma), float(cap))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.empty(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def gauss3(atom_id: int, step: int, seed: int):
    g = np.empty(3)
    lib().oracle_gauss3(int(atom_id), int(step), int(seed), _p(g))
    return g


def couple(v, mass_of_atom, A, T, chi, *, mode, frozen, seed, md_step, dt_md, gamma_fs, VC,
           stop_beta=0.0, stop_ecut=0.0, rng_id=None):
    """Hand-over of one MD step (oracle_couple); rng_id: int64 ids keying the
    atoms' Langevin numbers (None: the atom index)."""
    n = T.shape[0]
    dKE = np.empty(n)
    rid = None
    if rng_id is not None:
        rid = np.ascontiguousarray(rng_id, dtype=np.int64)
        assert rid.shape == (n,)
    stopped = lib().oracle_couple(n, _p(v), _p(mass_of_atom), _p(A), _p(T), _p(chi), int(mode),
                                  int(frozen), int(seed), int(md_step), float(dt_md),
                                  float(gamma_fs), float(VC), _p(dKE), float(stop_beta), float(stop_ecut),
                                  _p(rid) if rid is not None else None)
    return dKE, int(stopped)


def morse(r: float, D: float, alpha: float, r0: float):
    """(phi, phi') of the unshifted Morse pair potential [eV, eV/A]."""
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().oracle_morse(float(r), float(D), float(alpha), float(r0), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def forces(x, box, periodic, rowptr, col, *, D, alpha, r0, rc):
    """Shifted-force Morse forces [N, 3] (eV/A) and per-atom energies [N] (eV)."""
    q, Lq = quantize(x, box, periodic)
    n = x.shape[0]
    F = np.zeros((n, 3))
    E = np.zeros(n)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    lib().oracle_forces(n, _p(rowptr), _p(col), _p(q), _p(Lq), _p(per), float(D), float(alpha), float(r0),
                        float(rc), _p(F), _p(E))
    return F, E


def kick(v, F, mass_of_atom, dt: float):
    """v += dt F / m in place (velocity-Verlet half kick with dt = half the step)."""
    lib().oracle_kick(v.shape[0], _p(v), _p(F), _p(mass_of_atom), float(dt))


# --------------------------------------------------------------------------
# material law and derived per-step scalars (Sec. 2, Eq. Kij)

def ce_integral(T: np.ndarray, gamma: float, cap: float) -> np.ndarray:
    """int_0^T C_e(T') dT' per unit volume for C_e = min(gamma T, cap) [J m^-3]."""
    T = np.asarray(T, dtype=np.float64)
    if cap <= 0:
        return 0.5 * gamma * T * T
    Tc = cap / gamma
    return np.where(T <= Tc, 0.5 * gamma * T * T, 0.5 * cap * Tc + cap * (T - Tc))


def local_stability_rate(p: dict, nmax: int, Tlat: float, Tmin: float, Tmax_atoms: float, cap: float) -> float:
    """Rate bound [1/fs] of the LOCAL form's explicit step, 2 n_max K + G / C_min:
    in the energy variables U_i the linearised pair terms form a symmetric matrix
    whose rows sum to at most K = 2 d kappa_ij / (Z b^2 C_e) per pair (the step in
    T has the same spectrum: its Jacobian is similar to that one).  kappa_mode 1:
    K = 2 d kappa0 / (gamma Z b^2 T_lat), times T_hi / T_c where the hottest atom
    is above the cap; kappa_mode 0: K = 2 d kappa0 / (Z b^2 C_e(T_min))."""
    g = p["gamma_Ce"]
    def ce(T):
        c = g * T
        return min(c, cap) if cap > 0 else c
    geo = 2.0 * p["dim_d"] / (p["zb2"] * 1e-20)
    if p["kappa_mode"] == 1:
        K = geo * p["kappa0"] / (g * Tlat) if Tlat > 0 else float("inf")
        if cap > 0 and g * Tmax_atoms > cap:
            K *= Tmax_atoms / (cap / g)
    else:
        K = geo * p["kappa0"] / ce(Tmin) if Tmin > 0 else float("inf")
    cmin = ce(Tmin)
    return (2.0 * nmax * K + (p["G"] / cmin if cmin > 0 else float("inf"))) * 1e-15


class OracleSim:
    """MD-step driver around the oracle primitives, with the same call sequence
    as the library: set_te -> per MD step [build(x, v) -> substeps(n) ->
    couple(v, dt_md)] -> energy().  All arrays in original atom order, FP64.

    p: dict with keys rc, dt_sub, Tmax, gamma_Ce, Ce_cap_kB, kappa0,
    kappa_mode, G, eps_ke, dim_d, zb2, couple_mode, frozen, seed, dof_mode,
    vatom (<= 0: box volume / N), and optionally 'laser' (dict with
    fluence_Jm2, lp_A, t0_fs, sigma_fs) with `depth` per atom, and ce_mode
    (0: C_e and kappa_e at the system means, Sec. 2; 1: the LOCAL per-atom form,
    substeps_local, whose ledger is E_e = sum_i V_atom U(T_i)).
    """

    def __init__(self, p: dict, box, periodic, mass_amu, types, depth=None):
        self.p = dict(p)
        self.box = np.asarray(box, dtype=np.float64)
        self.per = np.asarray(periodic, dtype=np.int32)
        self.mass = np.asarray(mass_amu, dtype=np.float64)[np.asarray(types)]
        self.mass = np.ascontiguousarray(self.mass)
        self.n = self.mass.shape[0]
        v = self.p.get("vatom", 0.0)
        self.vatom = float(v) if v and v > 0 else float(np.prod(self.box)) / self.n
        self.depth = depth
        self.md_step = 0
        self.rng_ids = None   # ids keying the Langevin numbers (None: the atom index)
        self.T = None
        self.A = np.zeros(self.n)
        self.E_lat = 0.0
        self.E_src = 0.0
        self.n_stopped = 0
        self.VC = None
        self.Tfix = None          # border temperatures (NaN: free atom), original order
        self.E_res = 0.0          # energy absorbed by the border in closed MD steps [eV]
        self.eres_T = np.zeros(1) # kelvin sum absorbed in the current MD step
        self.E_res_local = 0.0    # border energy of the LOCAL form [eV]

    def set_border(self, Tfix):
        """Fixed-temperature border: atoms with a finite Tfix are held there."""
        self.Tfix = None if Tfix is None else np.ascontiguousarray(Tfix, dtype=np.float64).copy()

    # electronic temperature ------------------------------------------------
    def set_te(self, Te):
        self.T = np.ascontiguousarray(Te, dtype=np.float64).copy()
        cap = self.cap_SI()
        self.E_e0 = float((ce_integral(self.T, self.p["gamma_Ce"], cap)
                           * self.vatom * 1e-30 / EV_J).sum())
        self.E_base = self.E_e0
        self.ST_base = float(self.T.sum())

    def cap_SI(self) -> float:
        c = self.p.get("Ce_cap_kB", 0.0)
        return c * KB_J / (self.vatom * 1e-30) if c and c > 0 else 0.0

    # per MD step -------------------------------------------------------------
    def build(self, x, v):
        p = self.p
        if self.VC is not None:
            s = float(self.T.sum())
            self.E_base += self.VC * (s - self.ST_base)
            self.ST_base = s
            self.E_res += self.VC * float(self.eres_T[0])
            self.eres_T[0] = 0.0
        self.rowptr, self.col = neighbors(x, self.box, self.per, p["rc"])
        self.x_build = np.ascontiguousarray(x, dtype=np.float64).copy()
        ns = int(p.get("rate_shell_n", 0))
        self.w = pair_weights(x, self.box, self.per, self.rowptr, self.col, p["zb2"], ns) if ns > 0 else None
        self.Tl, self.Kself = lattice_temperature(self.rowptr, self.col, v, self.mass,
                                                  p.get("dof_mode", 0))
        self.chi = np.ascontiguousarray((self.Kself >= p["eps_ke"]).astype(np.uint8))
        # global means: mean electronic temperature and the classical lattice
        # temperature K / ((3/2) k_B N) (Sec. 2)
        Te_mean = float(self.T.mean())
        ke = 0.5 * self.mass * (v * v).sum(axis=1) * MVV_EV
        Tlat = float(ke.sum() / (1.5 * KB_EV * self.n))
        self.Tmin = float(self.T.min()) if self.n else 0.0
        self.Tmax_atoms = float(self.T.max()) if self.n else 0.0
        self.set_step_means(Te_mean, Tlat)

    def set_step_means(self, Te_mean: float, Tlat: float):
        """C_e, kappa_e, K and the coupling constants of the MD step from the
        system means (Sec. 2: evaluated at the mean electronic and lattice
        temperatures); a domain of a decomposed system passes the means of the
        whole system."""
        p = self.p
        self.Te_mean, self.Tlat = float(Te_mean), float(Tlat)
        Ce = p["gamma_Ce"] * self.Te_mean
        cap = self.cap_SI()
        if cap > 0:
            Ce = min(Ce, cap)
        kappa = p["kappa0"] * (self.Te_mean / self.Tlat if p["kappa_mode"] == 1 else 1.0)
        self.Ce = Ce
        self.K = 2.0 * p["dim_d"] * kappa / (Ce * p["zb2"] * 1e-20) * 1e-15
        self.cG = p["G"] / Ce * 1e-15
        self.VG = p["G"] * self.vatom * 1e-30 / EV_J * 1e-15
        self.VC = self.vatom * 1e-30 * Ce / EV_J
        self.gamma_L = p["G"] * self.vatom * 1e-30 / (3.0 * KB_J) * 1e-15
        nmax = int(np.diff(self.rowptr).max()) if self.n else 0
        self.stability = p["dt_sub"] * (2.0 * nmax * self.K + self.cG)
        if p.get("ce_mode", 0) == 1:
            self.stability = p["dt_sub"] * local_stability_rate(p, nmax, self.Tlat, self.Tmin,
                                                                 self.Tmax_atoms, cap)

    def substeps(self, n_sub: int, t_start: float = 0.0):
        if self.stability > 2.0:
            raise ValueError("unstable substep")
        p = self.p
        if p.get("ce_mode", 0) == 1:
            st, es, er = substeps_local(self.rowptr, self.col, self.T, self.Tl, self.chi, self.A, n_sub,
                                        p["dt_sub"], p["Tmax"], kappa0=p["kappa0"],
                                        kappa_mode=p["kappa_mode"], Tlat=self.Tlat, dim_d=p["dim_d"],
                                        S2_A2=p["zb2"], gamma=p["gamma_Ce"], cap_SI=self.cap_SI(),
                                        G=p["G"], vatom_A3=self.vatom, depth=self.depth,
                                        source=p.get("laser"), t_start=t_start, Tfix=self.Tfix,
                                        weights=self.w)
            if st < 0:
                raise FloatingPointError(f"theta left [0,1] at substep {-st - 1}")
            self.E_src += es
            self.E_res_local += er
            return
        st, es = substeps(self.rowptr, self.col, self.T, self.Tl, self.chi, self.A, n_sub,
                          p["dt_sub"], p["Tmax"], self.K, self.cG, self.VG, depth=self.depth,
                          source=p.get("laser"), Ce_SI=self.Ce, vatom_A3=self.vatom,
                          t_start=t_start, Tfix=self.Tfix, eres=self.eres_T, weights=self.w)
        if st < 0:
            raise FloatingPointError(f"theta left [0,1] at substep {-st - 1}")
        self.E_src += es

    def forces(self):
        """Shifted-force Morse forces and potential energy at the positions of the
        last build (p: pot_D, pot_alpha, pot_r0; cutoff rc)."""
        p = self.p
        F, E = forces(self.x_build, self.box, self.per, self.rowptr, self.col, D=p["pot_D"],
                      alpha=p["pot_alpha"], r0=p["pot_r0"], rc=p["rc"])
        return F, float(E.sum())

    def couple(self, v, dt_md: float):
        p = self.p
        local = p.get("ce_mode", 0) == 1
        if local:
            Tb, Ab = self.T.copy(), self.A.copy()
        dKE, stopped = couple(v, self.mass, self.A, self.T, self.chi, mode=p["couple_mode"],
                              frozen=p["frozen"], seed=p["seed"], md_step=self.md_step,
                              dt_md=dt_md, gamma_fs=self.gamma_L, VC=self.VC,
                              stop_beta=p.get("stop_beta", 0.0), stop_ecut=p.get("stop_ecut", 10.0),
                              rng_id=self.rng_ids)
        if local:
            # a stopped atom's unpaid energy returns to its own electrons: U_i += (A_i - dKE_i) / V
            idx = np.nonzero(self.T != Tb)[0]
            cap = self.cap_SI()
            for i in idx:
                U = ce_energy(Tb[i], p["gamma_Ce"], cap) + (Ab[i] - dKE[i]) * EV_J / (self.vatom * 1e-30)
                self.T[i] = ce_energy_inv(U, p["gamma_Ce"], cap)
        self.E_lat += float(dKE.sum())
        self.n_stopped += stopped
        self.md_step += 1
        return dKE

    def energy(self) -> dict:
        s = float(self.T.sum())
        E_e = self.E_base + self.VC * (s - self.ST_base) if self.VC is not None else self.E_base
        E_res = self.E_res + (self.VC * float(self.eres_T[0]) if self.VC is not None else 0.0)
        if self.p.get("ce_mode", 0) == 1:
            E_e = float((ce_integral(self.T, self.p["gamma_Ce"], self.cap_SI())
                         * self.vatom * 1e-30 / EV_J).sum())
            E_res = self.E_res_local
        return {"E_e": E_e, "E_lat": self.E_lat, "E_src": self.E_src, "E_e0": self.E_e0, "E_res": E_res,
                "sum_T": s, "max_T": float(self.T.max()),
                "drift": (E_e + self.E_lat - self.E_src + E_res - self.E_e0) / max(abs(self.E_e0), abs(E_e))}
