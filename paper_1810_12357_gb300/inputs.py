"""Seeded synthetic inputs for the electronic-heat-conduction path.

This module only builds inputs (atom positions, velocities, initial electronic
temperatures, material parameters).  It holds none of the method's arithmetic:
no neighbour search, no flux, no coupling.  Both the CPU oracle and the CUDA
library are fed from here, so the same seed gives the same system on both.

Units throughout: Angstrom, femtosecond, electron-volt, atomic mass unit, kelvin.

Workloads follow the systems of the paper: FCC metal lattices with periodic
boundaries (Sec. 3.2 bar, Sec. 4 cascade cell), a hot electronic region
(Sec. 3 hot zone, Sec. 4 cascade core), and a slab with free surfaces heated by
a laser pulse (Sec. 5, Eq. LaserIntesity).  Copper stands in for nickel with the
material constants listed in ``CU``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# CODATA 2018 exact / recommended values.
KB_EV = 8.617333262e-5            # Boltzmann constant [eV/K]
AMU_KG = 1.66053906660e-27        # atomic mass unit [kg]
EV_J = 1.602176634e-19            # electron-volt [J]
# kinetic-energy unit: 1 amu * (Angstrom/fs)^2 expressed in eV
AMU_A2_FS2_EV = AMU_KG * 1.0e10 / EV_J

CU_MASS_AMU = 63.546
CU_A = 3.615


@dataclasses.dataclass
class Material:
    """Electronic material law of the paper (Sec. 2): C_e = gamma*T_e,
    kappa_e = kappa0 (constant) or kappa0*T_e/T_lat, coupling constant G."""
    gamma_Ce: float = 96.6          # J m^-3 K^-2
    Ce_cap_kB: float = 0.0          # cap on C_e per atom in units of k_B (0: none)
    kappa0: float = 400.0           # W m^-1 K^-1
    kappa_mode: int = 0             # 0 constant, 1 kappa0*<T_e>/<T_l>
    G: float = 1.0e17               # W m^-3 K^-1


@dataclasses.dataclass
class System:
    """One atomistic system: positions x [N,3], velocities v [N,3], initial
    electronic temperature Te [N], box lengths, periodic flags, mass per atom
    type (one type here) and per-atom type index."""
    x: np.ndarray
    v: np.ndarray
    Te: np.ndarray
    box: np.ndarray
    periodic: np.ndarray
    mass_amu: np.ndarray
    type: np.ndarray
    a: float
    depth: np.ndarray | None = None   # distance below the irradiated surface [A]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def fcc_lattice(nx: int, ny: int, nz: int, a: float) -> np.ndarray:
    """Perfect FCC lattice of nx*ny*nz cubic cells with four-atom basis.
    Atom order: cell z slowest, then y, then x, then basis."""
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    return np.ascontiguousarray(pos)


def fcc_shell_vectors(a: float, rc: float) -> np.ndarray:
    """All ideal FCC lattice vectors r with 0 < |r| <= rc (geometry of the
    perfect crystal; used to state the lattice-sum parameters)."""
    m = int(math.ceil(rc / a)) + 1
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    out = []
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            for k in range(-m, m + 1):
                for b in basis:
                    r = (np.array([i, j, k], dtype=np.float64) + b) * a
                    d = math.sqrt(float(r @ r))
                    if 0.0 < d <= rc:
                        out.append(r)
    return np.array(out)


def fcc_shell_s2(a: float, rc: float) -> float:
    """Sum of |r|^2 over the ideal FCC neighbour shell inside rc.  For a
    nearest-neighbour cutoff this equals Z*b^2 of Eq. Kij (Z = 12, b = a/sqrt2)."""
    r = fcc_shell_vectors(a, rc)
    return float((r * r).sum())


def maxwell(n: int, T: float, mass_amu: float, rng: np.random.Generator) -> np.ndarray:
    """Maxwell-Boltzmann velocities [A/fs] at temperature T, global centre-of-mass
    velocity removed, not rescaled."""
    sig = math.sqrt(KB_EV * T / (mass_amu * AMU_A2_FS2_EV))
    v = rng.normal(0.0, sig, size=(n, 3))
    v -= v.mean(axis=0, keepdims=True)
    return np.ascontiguousarray(v)


def min_image(d: np.ndarray, box: np.ndarray, periodic: np.ndarray) -> np.ndarray:
    d = d.copy()
    for k in range(3):
        if periodic[k]:
            d[:, k] -= box[k] * np.round(d[:, k] / box[k])
    return d


def hot_spot(x: np.ndarray, box: np.ndarray, periodic: np.ndarray, center, peak: float,
             sigma: float, T0: float) -> np.ndarray:
    """T = T0 + (peak - T0) * exp(-|r - c|^2 / (2 sigma^2)), minimum image."""
    d = min_image(x - np.asarray(center, dtype=np.float64)[None, :], box, periodic)
    r2 = (d * d).sum(axis=1)
    return T0 + (peak - T0) * np.exp(-r2 / (2.0 * sigma * sigma))


def track(x: np.ndarray, box: np.ndarray, periodic: np.ndarray, peak: float, r0: float,
          T0: float) -> np.ndarray:
    """Swift-ion track: radial Gaussian about the z-axis through the (x, y) box
    centre, T = T0 + (peak - T0) exp(-rho^2 / (2 r0^2))."""
    c = np.array([0.5 * box[0], 0.5 * box[1], 0.0])
    d = min_image(x - c[None, :], box, periodic)
    rho2 = d[:, 0] ** 2 + d[:, 1] ** 2
    return T0 + (peak - T0) * np.exp(-rho2 / (2.0 * r0 * r0))


def _finish(x, v, Te, box, periodic, a, name, depth=None) -> System:
    n = x.shape[0]
    return System(x=np.ascontiguousarray(x, dtype=np.float64),
                  v=np.ascontiguousarray(v, dtype=np.float64),
                  Te=np.ascontiguousarray(Te, dtype=np.float64),
                  box=np.asarray(box, dtype=np.float64),
                  periodic=np.asarray(periodic, dtype=np.int32),
                  mass_amu=np.array([CU_MASS_AMU], dtype=np.float64),
                  type=np.zeros(n, dtype=np.int32), a=a, depth=depth, name=name)


def wrap(x: np.ndarray, box: np.ndarray, periodic: np.ndarray) -> np.ndarray:
    x = x.copy()
    for k in range(3):
        if periodic[k]:
            x[:, k] = np.mod(x[:, k], box[k])
    return x


def hot_spot_system(n_cells: int, seed: int, *, a: float = CU_A, disp_sigma: float = 0.05,
                    T_lat: float = 300.0, T0: float = 300.0, peak: float = 3000.0,
                    sigma: float = 8.0) -> System:
    """Periodic FCC Cu cube of n_cells^3 cells, Gaussian position noise,
    Maxwell velocities and a Gaussian electronic hot spot at the box centre."""
    rng = np.random.default_rng(seed)
    box = np.array([n_cells * a] * 3)
    per = np.array([1, 1, 1], dtype=np.int32)
    x = fcc_lattice(n_cells, n_cells, n_cells, a)
    if disp_sigma > 0:
        x = x + rng.normal(0.0, disp_sigma, size=x.shape)
    x = wrap(x, box, per)
    v = maxwell(x.shape[0], T_lat, CU_MASS_AMU, rng)
    Te = hot_spot(x, box, per, 0.5 * box, peak, sigma, T0)
    return _finish(x, v, Te, box, per, a, f"hotspot_{n_cells}c")


def track_system(n_cells: int, seed: int, *, a: float = CU_A, T_lat: float = 300.0,
                 T0: float = 300.0, peak: float = 20000.0, r0: float = 20.0,
                 disp_sigma: float = 0.0) -> System:
    """Swift-ion track cell: periodic FCC Cu cube, Maxwell velocities, radial
    Gaussian T_e about the z axis."""
    rng = np.random.default_rng(seed)
    box = np.array([n_cells * a] * 3)
    per = np.array([1, 1, 1], dtype=np.int32)
    x = fcc_lattice(n_cells, n_cells, n_cells, a)
    if disp_sigma > 0:
        x = wrap(x + rng.normal(0.0, disp_sigma, size=x.shape), box, per)
    v = maxwell(x.shape[0], T_lat, CU_MASS_AMU, rng)
    Te = track(x, box, per, peak, r0, T0)
    return _finish(x, v, Te, box, per, a, f"track_{n_cells}c")


def laser_slab_system(nxy: int, nz: int, seed: int, *, a: float = CU_A, vacuum: float = 50.0,
                      vacancy_frac: float = 0.02, T_lat: float = 300.0, T0: float = 300.0) -> System:
    """Slab with free z surfaces: FCC Cu nxy x nxy x nz cells, periodic in x, y,
    `vacuum` Angstrom of empty space on both z faces, a random fraction of
    lattice sites left empty.  `depth` is the distance of each atom below the
    initial top surface (max z)."""
    rng = np.random.default_rng(seed)
    x = fcc_lattice(nxy, nxy, nz, a)
    keep = np.ones(x.shape[0], dtype=bool)
    n_vac = int(round(vacancy_frac * x.shape[0]))
    if n_vac > 0:
        keep[rng.choice(x.shape[0], size=n_vac, replace=False)] = False
    x = x[keep]
    x[:, 2] += vacuum
    box = np.array([nxy * a, nxy * a, nz * a + 2.0 * vacuum])
    per = np.array([1, 1, 0], dtype=np.int32)
    v = maxwell(x.shape[0], T_lat, CU_MASS_AMU, rng)
    Te = np.full(x.shape[0], T0)
    depth = x[:, 2].max() - x[:, 2]
    return _finish(x, v, Te, box, per, a, f"laser_{nxy}x{nxy}x{nz}", depth=depth)


def batch_replicas(n_rep: int, seed: int, *, n_min: int = 8000, n_max: int = 500000,
                   a: float = CU_A, scale: float = 1.0) -> list[System]:
    """Independent cascade cells: atom counts log-uniform in [n_min, n_max]
    (cubic FCC, n = 4 c^3), each with a Gaussian hot spot at a uniformly random
    position, peak U(5000, 30000) K, sigma U(5, 15) A, 300 K lattice.
    `scale` < 1 shrinks every replica's atom count for quick tests."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_rep):
        n_r = math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * scale
        c = max(3, int(round((n_r / 4.0) ** (1.0 / 3.0))))
        peak = rng.uniform(5000.0, 30000.0)
        sig = rng.uniform(5.0, 15.0)
        sub = np.random.default_rng(int(rng.integers(1 << 62)))
        box = np.array([c * a] * 3)
        per = np.array([1, 1, 1], dtype=np.int32)
        x = fcc_lattice(c, c, c, a)
        v = maxwell(x.shape[0], 300.0, CU_MASS_AMU, sub)
        centre = sub.uniform(0.0, 1.0, size=3) * box
        Te = hot_spot(x, box, per, centre, peak, sig, 300.0)
        out.append(_finish(x, v, Te, box, per, a, f"replica_{r}"))
    return out


def random_box_system(n: int, box, seed: int, periodic=(1, 1, 1), T_lat: float = 300.0,
                      Te_lo: float = 300.0, Te_hi: float = 3000.0) -> System:
    """Uniformly random atoms in a box (for brute-force neighbour checks)."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    x = rng.uniform(0.0, 1.0, size=(n, 3)) * box[None, :]
    v = maxwell(n, T_lat, CU_MASS_AMU, rng)
    Te = rng.uniform(Te_lo, Te_hi, size=n)
    return _finish(x, v, Te, box, np.asarray(periodic, dtype=np.int32), CU_A, "random")


# --------------------------------------------------------------------------
# Run parameters of the workloads (plain data; every side converts units itself).
#   rc       neighbour cutoff [A] (inclusive)
#   dt_sub   electronic substep [fs]
#   Tmax     T_max of the normalisation theta = T / T_max (T_min = 0)
#   Tref     reference temperature of the single-precision mirror [K]
#   gamma_Ce, Ce_cap_kB, kappa0, kappa_mode, G: material law (Material)
#   eps_ke   kinetic-energy guard [eV] below which an atom does not couple
#   dim_d    dimension d of Eq. Kij; zb2 the Z b^2 of Eq. Kij [A^2]
#   couple_mode 0 damping, 1 Langevin; frozen 1 keeps velocities fixed
#   seed     Philox key; dof_mode 0: (3/2) k_B N_j divisor, 1: (3/2) k_B (N_j - 1)
#   vatom    atomic volume [A^3] (<= 0: box volume / N)
#   flux_prec 0 single-precision pair flux, 1 double precision

def params_hotspot_fp64(a: float = CU_A) -> dict:
    """4,000-atom hot spot, frozen atoms, double-precision flux."""
    return dict(rc=4.0, dt_sub=1.0e-3, Tmax=2.0e4, Tref=300.0, gamma_Ce=96.6, Ce_cap_kB=0.0,
                kappa0=400.0, kappa_mode=0, G=1.0e17, eps_ke=1.0e-5, dim_d=3,
                zb2=fcc_shell_s2(a, 4.0), couple_mode=0, frozen=1, seed=1, dof_mode=0,
                vatom=0.0, flux_prec=1)


def params_track(a: float = CU_A) -> dict:
    """Swift-ion track: C_e capped at 3 k_B per atom, kappa0 T_e/T_l, Langevin."""
    return dict(rc=4.0, dt_sub=1.0e-3, Tmax=1.0e5, Tref=300.0, gamma_Ce=96.6, Ce_cap_kB=3.0,
                kappa0=400.0, kappa_mode=1, G=1.0e17, eps_ke=1.0e-5, dim_d=3,
                zb2=fcc_shell_s2(a, 4.0), couple_mode=1, frozen=0, seed=2, dof_mode=0,
                vatom=0.0, flux_prec=0)


def params_laser(a: float = CU_A) -> dict:
    """Laser slab: as the track, plus a Gaussian pulse (100 fs FWHM, 0.1 J/cm^2
    absorbed, 15 nm penetration) peaking at t0 = 50 fs."""
    p = params_track(a)
    p.update(seed=3, vatom=a ** 3 / 4.0,
             laser=dict(fluence_Jm2=1000.0, lp_A=150.0, t0_fs=50.0,
                        sigma_fs=100.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))))
    return p
