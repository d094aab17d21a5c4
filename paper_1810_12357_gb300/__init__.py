"""Python binding of libehc (include/ehc.h): electronic heat conduction for
two-temperature molecular dynamics (Ullah & Ponga, arXiv 1810.12357) on one
GB300 GPU.

The binding only marshals arguments: every computation runs in the CUDA
kernels of ``libehc.so``.  PyTorch supplies device memory and the stream.
There is no CPU fallback: if the library or a GPU is missing, calls raise.

    from paper_1810_12357_gb300 import Ehc, inputs
    s = inputs.track_system(20, seed=2)
    sim = Ehc(inputs.params_track(), s)          # ehc_create
    sim.set_te(s.Te)                             # ehc_set_te
    sim.build_neighbors(x, v)                    # per MD step
    sim.substep(100, t_fs)
    sim.couple(v, 1.0)
    sim.energy()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libehc.so")

EHC_OK = 0
ERRORS = {-1: "INVAL", -2: "NOMEM", -3: "CUDA", -4: "UNSTABLE", -5: "RANGE", -6: "NBR_OVERFLOW",
          -7: "TIMEOUT", -8: "STATE", -9: "BOUNDS"}


class EhcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.ehc_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})")


class ehc_params(ctypes.Structure):
    _fields_ = [
        ("rc_A", ctypes.c_double), ("dt_sub_fs", ctypes.c_double), ("Tmax_K", ctypes.c_double),
        ("Tref_K", ctypes.c_double), ("gamma_Ce", ctypes.c_double), ("Ce_cap_kB", ctypes.c_double),
        ("kappa0", ctypes.c_double), ("G", ctypes.c_double), ("eps_ke_eV", ctypes.c_double),
        ("zb2_A2", ctypes.c_double), ("vatom_A3", ctypes.c_double),
        ("laser_fluence_Jm2", ctypes.c_double), ("laser_lp_A", ctypes.c_double),
        ("laser_t0_fs", ctypes.c_double), ("laser_sigma_fs", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("dim_d", ctypes.c_int32), ("kappa_mode", ctypes.c_int32),
        ("couple_mode", ctypes.c_int32), ("frozen", ctypes.c_int32), ("dof_mode", ctypes.c_int32),
        ("flux_prec", ctypes.c_int32), ("laser_on", ctypes.c_int32), ("max_neighbors", ctypes.c_int32),
        ("use_graph", ctypes.c_int32), ("tile_threads", ctypes.c_int32), ("rate_shell_n", ctypes.c_int32),
        ("ce_mode", ctypes.c_int32), ("tile_grid_quarters", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
        ("pot_D_eV", ctypes.c_double), ("pot_alpha_perA", ctypes.c_double), ("pot_r0_A", ctypes.c_double),
        ("stop_beta_per_fs", ctypes.c_double), ("stop_ecut_eV", ctypes.c_double), ("skin_A", ctypes.c_double),
    ]


class ehc_energy_t(ctypes.Structure):
    _fields_ = [
        ("E_e", ctypes.c_double), ("E_lat", ctypes.c_double), ("E_src", ctypes.c_double),
        ("E_e0", ctypes.c_double), ("drift", ctypes.c_double), ("sum_T", ctypes.c_double),
        ("max_T", ctypes.c_double), ("mean_T", ctypes.c_double), ("Te_mean_step", ctypes.c_double),
        ("Tlat_step", ctypes.c_double), ("Ce_SI", ctypes.c_double), ("K_per_fs", ctypes.c_double),
        ("stability", ctypes.c_double), ("n_stopped", ctypes.c_int64), ("md_step", ctypes.c_int64),
        ("max_count", ctypes.c_int32), ("device_error", ctypes.c_int32), ("E_res", ctypes.c_double),
    ]


# every entry point of include/ehc.h with its ctypes signature
_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "ehc_create": (_I, [ctypes.POINTER(ehc_params), ctypes.c_int64, _P, _P, _P, ctypes.c_int32, _P, _P,
                        ctypes.POINTER(_P)]),
    "ehc_set_te": (_I, [_P, _P]),
    "ehc_set_depth": (_I, [_P, _P]),
    "ehc_set_border": (_I, [_P, _P]),
    "ehc_build_neighbors": (_I, [_P, _P, _P]),
    "ehc_substep": (_I, [_P, ctypes.c_int32, ctypes.c_double]),
    "ehc_couple": (_I, [_P, _P, ctypes.c_double]),
    "ehc_drift": (_I, [_P, _P, _P, ctypes.c_double]),
    "ehc_forces": (_I, [_P, _P, ctypes.POINTER(ctypes.c_double)]),
    "ehc_kick": (_I, [_P, _P, _P, ctypes.c_double]),
    "ehc_max_speed": (_I, [_P, _P, ctypes.POINTER(ctypes.c_double)]),
    "ehc_probe_wait": (_I, [_P, ctypes.c_uint32, ctypes.c_int32]),
    "ehc_get_te_at": (_I, [_P, _P, ctypes.c_int64, _P]),
    "ehc_set_te_at": (_I, [_P, _P, ctypes.c_int64, _P]),
    "ehc_set_step_means": (_I, [_P, ctypes.c_double, ctypes.c_double]),
    "ehc_set_rng_ids": (_I, [_P, _P, ctypes.c_int64]),
    "ehc_sums_at": (_I, [_P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]),
    "ehc_md_step_host": (_I, [_P, _P, _P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _P]),
    "ehc_energy": (_I, [_P, ctypes.POINTER(ehc_energy_t)]),
    "ehc_sync": (_I, [_P]),
    "ehc_get_te": (_I, [_P, _P]),
    "ehc_get_lattice_temperature": (_I, [_P, _P]),
    "ehc_export_neighbors": (_I, [_P, _P, _P, ctypes.c_int64]),
    "ehc_philox_normals": (_I, [_P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, _P, _P]),
    "ehc_save": (_I, [_P, ctypes.c_char_p]),
    "ehc_load": (_I, [_P, ctypes.c_char_p]),
    "ehc_electron_energy_noalloc": (_I, [_P, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _P, _P]),
    "ehc_nn_create": (_I, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(_P)]),
    "ehc_nn_set_params": (_I, [_P, _P, _P]),
    "ehc_nn_get_params": (_I, [_P, _P, _P]),
    "ehc_nn_train_step": (_I, [_P, _P, _P, _P, ctypes.c_float, _P, _P]),
    "ehc_nn_predict": (_I, [_P, _P, _P, _P]),
    "ehc_nn_step": (_I, [_P, _P, ctypes.c_double, ctypes.c_double, _P, _P]),
    "ehc_nn_destroy": (None, [_P]),
    "ehc_cheb_create": (_I, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                             ctypes.POINTER(_P)]),
    "ehc_cheb_coefficients": (_I, [_P, _P, _P, _P, _P]),
    "ehc_cheb_step": (_I, [_P, _P, ctypes.c_double, ctypes.c_double, _P, _P]),
    "ehc_cheb_stats": (_I, [_P, _P, _P]),
    "ehc_cheb_set_coefficients": (_I, [_P, _P, _P, _P, _P, _P]),
    "ehc_cheb_train_step": (_I, [_P, _P, _P, _P, ctypes.c_float, ctypes.c_int32, _P, _P]),
    "ehc_cheb_predict": (_I, [_P, _P, _P, _P]),
    "ehc_cheb_train_rollout": (_I, [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_float, ctypes.c_int32, _P, _P]),
    "ehc_cheb_stability": (_I, [_P, _P]),
    "ehc_cheb_spectrum": (_I, [_P, _P, _P, ctypes.c_int32, _P]),
    "ehc_cheb_destroy": (None, [_P]),
    "ehc_cheb_set_corrector": (_I, [_P, _P]),
    "ehc_tuning": (_I, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "ehc_batch_tuning": (_I, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "ehc_gnn_create": (_I, [_P, ctypes.c_double, ctypes.POINTER(_P)]),
    "ehc_gnn_set_params": (_I, [_P, _P, _P]),
    "ehc_gnn_get_params": (_I, [_P, _P, _P]),
    "ehc_gnn_apply": (_I, [_P, _P, ctypes.c_double, _P, _P, _P]),
    "ehc_gnn_train_step": (_I, [_P, _P, ctypes.c_double, _P, _P, ctypes.c_float, _P, _P]),
    "ehc_gnn_destroy": (None, [_P]),
    "ehc_batch_create": (_I, [ctypes.POINTER(ehc_params), ctypes.c_int32, _P, _P, _P, _P, _P,
                              ctypes.POINTER(_P)]),
    "ehc_batch_size": (_I, [_P, _P, _P]),
    "ehc_batch_set_te": (_I, [_P, _P]),
    "ehc_batch_build_neighbors": (_I, [_P, _P, _P]),
    "ehc_batch_substep": (_I, [_P, ctypes.c_int32, ctypes.c_double]),
    "ehc_batch_couple": (_I, [_P, _P, ctypes.c_double]),
    "ehc_batch_drift": (_I, [_P, _P, _P, ctypes.c_double]),
    "ehc_batch_get_te": (_I, [_P, _P]),
    "ehc_batch_energy": (_I, [_P, ctypes.c_int32, ctypes.POINTER(ehc_energy_t)]),
    "ehc_batch_destroy": (None, [_P]),
    "ehc_destroy": (None, [_P]),
    "ehc_strerror": (ctypes.c_char_p, [_I]),
}

_lib = None


def load_library(path: str | None = None):
    """Load libehc.so (raises if it has not been built: no fallback exists).
    With EHC_CHECKED=1 in the environment the bounds-checked build
    libehc_checked.so is loaded instead (build.build(checked=True) makes it)."""
    global _lib
    if _lib is None:
        p = path or (os.path.join(os.path.dirname(LIB_PATH), "libehc_checked.so")
                     if os.environ.get("EHC_CHECKED") == "1" else LIB_PATH)
        if not os.path.exists(p):
            raise RuntimeError(f"libehc.so not built ({p}); run __graft_entry__.build()")
        L = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != EHC_OK:
        raise EhcError(code, where)


def make_params(p: dict) -> ehc_params:
    """Marshal a parameter dict (see inputs.params_*) into the C struct."""
    q = ehc_params()
    q.rc_A = p["rc"]
    q.dt_sub_fs = p["dt_sub"]
    q.Tmax_K = p["Tmax"]
    q.Tref_K = p.get("Tref", 300.0)
    q.gamma_Ce = p["gamma_Ce"]
    q.Ce_cap_kB = p.get("Ce_cap_kB", 0.0)
    q.kappa0 = p["kappa0"]
    q.G = p["G"]
    q.eps_ke_eV = p["eps_ke"]
    q.zb2_A2 = p["zb2"]
    q.vatom_A3 = p.get("vatom", 0.0)
    las = p.get("laser")
    if las:
        q.laser_on = 1
        q.laser_fluence_Jm2 = las["fluence_Jm2"]
        q.laser_lp_A = las["lp_A"]
        q.laser_t0_fs = las["t0_fs"]
        q.laser_sigma_fs = las["sigma_fs"]
    q.seed = int(p.get("seed", 0))
    q.dim_d = int(p["dim_d"])
    q.kappa_mode = int(p["kappa_mode"])
    q.couple_mode = int(p["couple_mode"])
    q.frozen = int(p["frozen"])
    q.dof_mode = int(p.get("dof_mode", 0))
    q.flux_prec = int(p.get("flux_prec", 0))
    q.max_neighbors = int(p.get("max_neighbors", 0))
    q.rate_shell_n = int(p.get("rate_shell_n", 0))
    q.ce_mode = int(p.get("ce_mode", 0))
    q.pot_D_eV = float(p.get("pot_D", 0.0))
    q.pot_alpha_perA = float(p.get("pot_alpha", 0.0))
    q.pot_r0_A = float(p.get("pot_r0", 0.0))
    q.stop_beta_per_fs = float(p.get("stop_beta", 0.0))
    q.stop_ecut_eV = float(p.get("stop_ecut", 10.0))
    q.use_graph = int(p.get("use_graph", 1))
    q.tile_threads = int(p.get("tile_threads", 0))
    q.skin_A = float(p.get("skin", 0.0))
    q.tile_grid_quarters = int(p.get("tile_grid_quarters", 0))
    return q


def _ptr(t) -> int:
    import torch
    if t is None:
        return None
    assert t.is_contiguous(), "tensors passed to libehc must be contiguous"
    return ctypes.c_void_p(t.data_ptr())


def _stream() -> int:
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Ehc:
    """One system behind an ehc_ctx.  Arrays are torch tensors (float64,
    original atom order) on the CUDA device, or numpy arrays that are copied
    to the device first."""

    def __init__(self, params: dict, system=None, *, n=None, box=None, periodic=None, mass_amu=None,
                 types=None, device="cuda", tune_cache: bool = False):
        import torch
        L = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("libehc needs a CUDA device; there is no CPU path")
        self.device = torch.device(device)
        if system is not None:
            n, box, periodic, mass_amu, types = (system.n, system.box, system.periodic, system.mass_amu,
                                                 system.type)
        self.n = int(n)
        params = dict(params)
        # tune_cache: the row-tile choice stored for this GPU and shape (tuning.py),
        # else the tuner's choice is stored after the first long substep call
        self._tune_key = None
        if tune_cache and not params.get("tile_threads"):
            from . import tuning
            key = tuning.shape_class(self.n, box, params["rc"], params.get("skin", 0.0))
            got = tuning.lookup(key)
            if got:
                params["tile_threads"], params["tile_grid_quarters"] = got
            else:
                self._tune_key = key
        self.params = params
        self._p = make_params(params)
        box_a = np.ascontiguousarray(box, dtype=np.float64)
        per_a = np.ascontiguousarray(periodic, dtype=np.int32)
        m_a = np.ascontiguousarray(mass_amu, dtype=np.float64)
        self._types = None
        nt = int(m_a.shape[0])
        if nt > 1:
            self._types = torch.as_tensor(np.asarray(types, dtype=np.int32), device=self.device).contiguous()
        h = ctypes.c_void_p()
        _check(L.ehc_create(ctypes.byref(self._p), self.n, box_a.ctypes.data_as(_P), per_a.ctypes.data_as(_P),
                            m_a.ctypes.data_as(_P), nt, _ptr(self._types) if self._types is not None else None,
                            _stream(), ctypes.byref(h)), "ehc_create")
        self._h = h
        self._lib = L

    # ---------------------------------------------------------------- helpers
    def _dev(self, a):
        import torch
        if isinstance(a, torch.Tensor):
            t = a if a.device == self.device else a.to(self.device)
            return t.to(torch.float64).contiguous()
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=self.device)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.ehc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- C-ABI calls
    def set_te(self, Te):
        t = self._dev(Te)
        _check(self._lib.ehc_set_te(self._h, _ptr(t)), "ehc_set_te")

    def set_depth(self, depth):
        t = self._dev(depth)
        _check(self._lib.ehc_set_depth(self._h, _ptr(t)), "ehc_set_depth")

    def set_border(self, Tfix):
        """Fixed-temperature border from the next build: atoms with a finite
        Tfix (caller order) are held there, NaN marks free atoms; None removes it."""
        if Tfix is None:
            _check(self._lib.ehc_set_border(self._h, None), "ehc_set_border")
            return
        t = self._dev(Tfix)
        _check(self._lib.ehc_set_border(self._h, _ptr(t)), "ehc_set_border")

    def build_neighbors(self, x, v):
        _check(self._lib.ehc_build_neighbors(self._h, _ptr(x), _ptr(v)), "ehc_build_neighbors")

    def substep(self, n_sub: int, t_fs: float = 0.0):
        _check(self._lib.ehc_substep(self._h, int(n_sub), float(t_fs)), "ehc_substep")
        if self._tune_key is not None:
            nt, q = self.tuning()
            if nt:
                from . import tuning
                tuning.store(self._tune_key, nt, q)
                self._tune_key = None

    def tuning(self):
        """(tile_threads, grid_quarters) the row-tile kernel runs with ((0, 0) before
        the first long substep call when tuned)."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.ehc_tuning(self._h, ctypes.byref(a), ctypes.byref(b)), "ehc_tuning")
        return a.value, b.value

    def couple(self, v, dt_md_fs: float):
        _check(self._lib.ehc_couple(self._h, _ptr(v), float(dt_md_fs)), "ehc_couple")

    def drift(self, x, v, dt_fs: float):
        _check(self._lib.ehc_drift(self._h, _ptr(x), _ptr(v), float(dt_fs)), "ehc_drift")

    def forces(self, F=None, energy: bool = True):
        """Morse forces of the last build's positions (caller order, [N, 3] eV/A) and
        the potential energy [eV] (None, without a synchronisation, if not `energy`)."""
        import torch
        if F is None:
            F = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        e = ctypes.c_double()
        _check(self._lib.ehc_forces(self._h, _ptr(F), ctypes.byref(e) if energy else None), "ehc_forces")
        return F, (e.value if energy else None)

    def kick(self, v, F, dt_fs: float):
        """v += dt F / m in place."""
        _check(self._lib.ehc_kick(self._h, _ptr(v), _ptr(F), float(dt_fs)), "ehc_kick")

    def get_te_at(self, idx, out=None):
        """T_e of the caller-order atoms idx (int32 device tensor) into a new or given tensor."""
        import torch
        if out is None:
            out = torch.empty(idx.numel(), dtype=torch.float64, device="cuda")
        _check(self._lib.ehc_get_te_at(self._h, _ptr(idx), int(idx.numel()), _ptr(out)), "ehc_get_te_at")
        return out

    def set_te_at(self, idx, vals):
        _check(self._lib.ehc_set_te_at(self._h, _ptr(idx), int(idx.numel()), _ptr(vals)), "ehc_set_te_at")

    def sums_at(self, idx):
        """(sum T_e, sum of the kinetic energy [eV]) over the caller-order atoms idx."""
        out = (ctypes.c_double * 2)()
        _check(self._lib.ehc_sums_at(self._h, _ptr(idx), int(idx.numel()), out), "ehc_sums_at")
        return out[0], out[1]

    def set_step_means(self, Te_mean: float, Tlat: float):
        _check(self._lib.ehc_set_step_means(self._h, float(Te_mean), float(Tlat)), "ehc_set_step_means")

    def set_rng_ids(self, ids, md_step: int):
        """Key the Langevin stream of the caller-order atoms by ids (int64 device
        tensor of n ids, or None for the caller index) and set the MD step counter."""
        if ids is not None:
            import torch
            ids = torch.as_tensor(ids).to(device=self.device, dtype=torch.int64).contiguous()
            if ids.numel() != self.n:
                raise ValueError("one id per atom")
        self._rng_ids = ids   # kept alive until the asynchronous copy has run
        _check(self._lib.ehc_set_rng_ids(self._h, _ptr(ids) if ids is not None else None, int(md_step)),
               "ehc_set_rng_ids")

    def probe_wait(self, polls: int, complete: bool) -> int:
        """Return code of the bounded-wait probe (EHC_E_TIMEOUT when it ran out)."""
        return int(self._lib.ehc_probe_wait(self._h, int(polls), 1 if complete else 0))

    def max_speed(self, v) -> float:
        r = ctypes.c_double()
        _check(self._lib.ehc_max_speed(self._h, _ptr(v), ctypes.byref(r)), "ehc_max_speed")
        return r.value

    def md_step_host(self, x_host, v_host, n_sub: int, t_fs: float, dt_md_fs: float, Te_host_out):
        """Whole MD step on host buffers (torch CPU tensors, ideally pinned)."""
        _check(self._lib.ehc_md_step_host(self._h, ctypes.c_void_p(x_host.data_ptr()),
                                          ctypes.c_void_p(v_host.data_ptr()), int(n_sub), float(t_fs),
                                          float(dt_md_fs), ctypes.c_void_p(Te_host_out.data_ptr())),
               "ehc_md_step_host")

    def energy(self, check: bool = True) -> dict:
        e = ehc_energy_t()
        code = self._lib.ehc_energy(self._h, ctypes.byref(e))
        if check:
            _check(code, "ehc_energy")
        d = {f: getattr(e, f) for f, _ in ehc_energy_t._fields_}
        d["status"] = code
        return d

    def sync(self):
        _check(self._lib.ehc_sync(self._h), "ehc_sync")

    def get_te(self):
        import torch
        out = torch.empty(self.n, dtype=torch.float64, device=self.device)
        _check(self._lib.ehc_get_te(self._h, _ptr(out)), "ehc_get_te")
        return out

    def get_lattice_temperature(self):
        import torch
        out = torch.empty(self.n, dtype=torch.float64, device=self.device)
        _check(self._lib.ehc_get_lattice_temperature(self._h, _ptr(out)), "ehc_get_lattice_temperature")
        return out

    def export_neighbors(self, cap_per_atom: int = 64):
        rowptr = np.zeros(self.n + 1, dtype=np.int64)
        col = np.empty(max(1, self.n * cap_per_atom), dtype=np.int32)
        _check(self._lib.ehc_export_neighbors(self._h, rowptr.ctypes.data_as(_P), col.ctypes.data_as(_P),
                                              col.shape[0]), "ehc_export_neighbors")
        return rowptr, col[: rowptr[-1]].copy()

    def save(self, path: str):
        _check(self._lib.ehc_save(self._h, path.encode()), "ehc_save")

    def load(self, path: str):
        _check(self._lib.ehc_load(self._h, path.encode()), "ehc_load")


def philox_normals(ids, md_step: int, seed: int):
    """Three standard normals per id from the Langevin Philox stream (device)."""
    import torch
    L = load_library()
    ids_t = torch.as_tensor(np.asarray(ids, dtype=np.int64), device="cuda")
    out = torch.empty((ids_t.shape[0], 3), dtype=torch.float64, device="cuda")
    _check(L.ehc_philox_normals(_ptr(ids_t), ids_t.shape[0], int(md_step), int(seed), _ptr(out), _stream()),
           "ehc_philox_normals")
    return out


def electron_energy_noalloc(Te, gamma_Ce: float, Ce_cap_kB: float, vatom_A3: float, out=None):
    """ehc_electron_energy_noalloc: (sum T, max T, E_e0 [eV]) of device temperatures
    without any device allocation by the library.  `out` (3 float64 on the device)
    is the caller's; it is created here only when not given."""
    import torch
    L = load_library()
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=Te.device)
    _check(L.ehc_electron_energy_noalloc(_ptr(Te), int(Te.numel()), float(gamma_Ce), float(Ce_cap_kB),
                                         float(vatom_A3), _ptr(out), _stream()), "ehc_electron_energy_noalloc")
    return out


class EhcBatch:
    """Independent replicas advanced together (ehc_batch_*).  `systems` is a
    list of inputs.System sharing one parameter set; per-atom arrays are the
    replicas' arrays concatenated in order (see `offsets`)."""

    def __init__(self, params: dict, systems, tune_cache: bool = False):
        import torch
        L = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("libehc needs a CUDA device; there is no CPU path")
        self._lib = L
        params = dict(params)
        self._tune_key = None
        if tune_cache and not params.get("tile_threads"):
            from . import tuning
            key = tuning.shape_class(sum(int(x.n) for x in systems), systems[0].box, params["rc"],
                                     params.get("skin", 0.0), replicas=len(systems))
            got = tuning.lookup(key)
            if got:
                params["tile_threads"], params["tile_grid_quarters"] = got
            else:
                self._tune_key = key
        self.params = params
        self._p = make_params(params)
        n = np.ascontiguousarray([s.n for s in systems], dtype=np.int64)
        boxes = np.ascontiguousarray(np.concatenate([s.box for s in systems]), dtype=np.float64)
        per = np.ascontiguousarray(systems[0].periodic, dtype=np.int32)
        m = np.ascontiguousarray(systems[0].mass_amu[:1], dtype=np.float64)
        h = ctypes.c_void_p()
        _check(L.ehc_batch_create(ctypes.byref(self._p), len(systems), n.ctypes.data_as(_P),
                                  boxes.ctypes.data_as(_P), per.ctypes.data_as(_P), m.ctypes.data_as(_P),
                                  _stream(), ctypes.byref(h)), "ehc_batch_create")
        self._h = h
        self.n_rep = len(systems)
        tot = ctypes.c_int64()
        off = np.zeros(self.n_rep, dtype=np.int64)
        _check(L.ehc_batch_size(h, ctypes.byref(tot), off.ctypes.data_as(_P)), "ehc_batch_size")
        self.n = int(tot.value)
        self.offsets = off

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.ehc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_te(self, Te):
        _check(self._lib.ehc_batch_set_te(self._h, _ptr(Te)), "ehc_batch_set_te")

    def build_neighbors(self, x, v):
        _check(self._lib.ehc_batch_build_neighbors(self._h, _ptr(x), _ptr(v)), "ehc_batch_build_neighbors")

    def substep(self, n_sub: int, t_fs: float = 0.0):
        _check(self._lib.ehc_batch_substep(self._h, int(n_sub), float(t_fs)), "ehc_batch_substep")
        if self._tune_key is not None:
            nt, q = self.tuning()
            if nt:
                from . import tuning
                tuning.store(self._tune_key, nt, q)
                self._tune_key = None

    def tuning(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.ehc_batch_tuning(self._h, ctypes.byref(a), ctypes.byref(b)), "ehc_batch_tuning")
        return a.value, b.value

    def couple(self, v, dt_md_fs: float):
        _check(self._lib.ehc_batch_couple(self._h, _ptr(v), float(dt_md_fs)), "ehc_batch_couple")

    def drift(self, x, v, dt_fs: float):
        _check(self._lib.ehc_batch_drift(self._h, _ptr(x), _ptr(v), float(dt_fs)), "ehc_batch_drift")

    def get_te(self):
        import torch
        out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(self._lib.ehc_batch_get_te(self._h, _ptr(out)), "ehc_batch_get_te")
        return out

    def energy(self, r: int) -> dict:
        e = ehc_energy_t()
        _check(self._lib.ehc_batch_energy(self._h, int(r), ctypes.byref(e)), "ehc_batch_energy")
        return {f: getattr(e, f) for f, _ in ehc_energy_t._fields_}


GNN_PARAMS = 6336   # parameters of the corrector network (include/ehc.h)


class EhcGnn:
    """Learned corrector of the window propagator (ehc_gnn_*): a message-passing
    network of node width 64 whose pair-flux output is added to a window's result.
    Bound to the atom count of the context it is created on; `ctx` arguments
    (default that context) supply the neighbour list and lattice temperatures."""

    def __init__(self, ctx: "Ehc", sigma: float = 1e-3, params=None):
        L = load_library()
        self._lib = L
        self.ctx = ctx
        self.sigma = float(sigma)
        h = ctypes.c_void_p()
        _check(L.ehc_gnn_create(ctx._h, self.sigma, ctypes.byref(h)), "ehc_gnn_create")
        self._h = h
        if params is not None:
            self.set_params(params)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.ehc_gnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        if a.shape != (GNN_PARAMS,):
            raise ValueError(f"the corrector takes {GNN_PARAMS} parameters")
        _check(self._lib.ehc_gnn_set_params(self._h, self.ctx._h, a.ctypes.data_as(_P)), "ehc_gnn_set_params")

    def get_params(self):
        a = np.empty(GNN_PARAMS, dtype=np.float32)
        _check(self._lib.ehc_gnn_get_params(self._h, self.ctx._h, a.ctypes.data_as(_P)), "ehc_gnn_get_params")
        return a

    def apply(self, Y, kappa: float, ctx=None, want_dY: bool = False):
        """Corrected result Y^ of Y (caller order, device FP64); with want_dY also
        the correction Y^ - Y."""
        import torch
        c = ctx or self.ctx
        out = torch.empty_like(Y)
        dY = torch.empty_like(Y) if want_dY else None
        _check(self._lib.ehc_gnn_apply(self._h, c._h, float(kappa), _ptr(Y), _ptr(out),
                                       _ptr(dY) if dY is not None else None), "ehc_gnn_apply")
        return (out, dY) if want_dY else out

    def train_step(self, Y, Tstar, kappa: float, lr: float, want_grad: bool = False, ctx=None):
        """Loss of the window Y -> T* and (lr > 0) one Adam step; with want_grad
        also the gradient [6336]."""
        c = ctx or self.ctx
        loss = ctypes.c_float()
        g = np.empty(GNN_PARAMS, dtype=np.float32) if want_grad else None
        _check(self._lib.ehc_gnn_train_step(self._h, c._h, float(kappa), _ptr(Y), _ptr(Tstar), float(lr),
                                            ctypes.byref(loss), g.ctypes.data_as(_P) if g is not None else None),
               "ehc_gnn_train_step")
        return (float(loss.value), g) if want_grad else float(loss.value)


class EhcNN:
    """Learned window propagator bound to a context (ehc_nn_*)."""

    def __init__(self, ctx: "Ehc", hidden: int = 8, n_window: int = 16, sigma: float = 1e-3, params=None):
        L = load_library()
        self._lib = L
        self.ctx = ctx
        self.H = int(hidden)
        self.n_window = int(n_window)
        self.sigma = float(sigma)
        self.np = 8 * self.H + 1
        h = ctypes.c_void_p()
        _check(L.ehc_nn_create(ctx._h, self.H, self.n_window, self.sigma, ctypes.byref(h)), "ehc_nn_create")
        self._h = h
        if params is not None:
            self.set_params(params)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.ehc_nn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        assert a.shape == (self.np,)
        _check(self._lib.ehc_nn_set_params(self._h, self.ctx._h, a.ctypes.data_as(_P)), "ehc_nn_set_params")

    def get_params(self):
        a = np.empty(self.np, dtype=np.float32)
        _check(self._lib.ehc_nn_get_params(self._h, self.ctx._h, a.ctypes.data_as(_P)), "ehc_nn_get_params")
        return a

    def train_step(self, Tin, Ttar, lr: float, want_grad: bool = False, ctx=None):
        """One Adam step on a window; `ctx` (same atom count) supplies the
        neighbour list and K, default the context the network was created on."""
        loss = ctypes.c_float()
        g = np.empty(self.np, dtype=np.float32) if want_grad else None
        c = ctx if ctx is not None else self.ctx
        _check(self._lib.ehc_nn_train_step(self._h, c._h, _ptr(Tin), _ptr(Ttar), ctypes.c_float(lr),
                                           ctypes.byref(loss), g.ctypes.data_as(_P) if g is not None else None),
               "ehc_nn_train_step")
        return (float(loss.value), g) if want_grad else float(loss.value)

    def predict(self, Tin):
        import torch
        out = torch.empty_like(Tin)
        _check(self._lib.ehc_nn_predict(self._h, self.ctx._h, _ptr(Tin), _ptr(out)), "ehc_nn_predict")
        return out

    def step(self, tau: float, t_fs: float = 0.0):
        fb = ctypes.c_int32()
        rho = ctypes.c_double()
        _check(self._lib.ehc_nn_step(self._h, self.ctx._h, float(tau), float(t_fs), ctypes.byref(fb),
                                     ctypes.byref(rho)), "ehc_nn_step")
        return bool(fb.value), float(rho.value)


class EhcCheb:
    """Chebyshev window propagator bound to a context (ehc_cheb_*)."""

    def __init__(self, ctx: "Ehc", n_window: int = 16, stages: int = 4, damping: float = 0.05, order: int = 1):
        L = load_library()
        self._lib = L
        self.ctx = ctx
        self.n_window = int(n_window)
        self.stages = int(stages)
        self.order = int(order)
        h = ctypes.c_void_p()
        _check(L.ehc_cheb_create(ctx._h, self.n_window, self.stages, self.order, float(damping), ctypes.byref(h)),
               "ehc_cheb_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.ehc_cheb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coefficients(self):
        """(nu, mut, kap, gam) for stages 0..s (index 0 unused)."""
        a = [np.empty(self.stages + 1) for _ in range(4)]
        _check(self._lib.ehc_cheb_coefficients(self._h, *[x.ctypes.data_as(_P) for x in a]),
               "ehc_cheb_coefficients")
        return tuple(a)

    def step(self, tau: float, t_fs: float = 0.0):
        fb = ctypes.c_int32()
        rho = ctypes.c_double()
        _check(self._lib.ehc_cheb_step(self._h, self.ctx._h, float(tau), float(t_fs), ctypes.byref(fb),
                                       ctypes.byref(rho)), "ehc_cheb_step")
        return bool(fb.value), float(rho.value)

    def stats(self):
        w = ctypes.c_int64()
        f = ctypes.c_int64()
        _check(self._lib.ehc_cheb_stats(self._h, ctypes.byref(w), ctypes.byref(f)), "ehc_cheb_stats")
        return int(w.value), int(f.value)

    def set_corrector(self, gnn):
        """Apply the corrector network (EhcGnn, or None) to every window's result."""
        _check(self._lib.ehc_cheb_set_corrector(self._h, gnn._h if gnn is not None else None),
               "ehc_cheb_set_corrector")
        self._corrector = gnn   # keep it alive while the window uses it

    def kappa(self, ctx=None) -> float:
        """n_w dt_sub K of the context's current MD step (the corrector's scale)."""
        c = ctx or self.ctx
        return self.n_window * c.params["dt_sub"] * c.energy(check=False)["K_per_fs"]

    def set_coefficients(self, nu, mut, kap, gam):
        """Replace the stage coefficients (arrays of stages + 1, index 0 unused);
        they become the base that training changes relatively."""
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (nu, mut, kap, gam)]
        if any(x.shape != (self.stages + 1,) for x in a):
            raise ValueError("coefficient arrays need stages + 1 entries")
        _check(self._lib.ehc_cheb_set_coefficients(self._h, self.ctx._h, *[x.ctypes.data_as(_P) for x in a]),
               "ehc_cheb_set_coefficients")

    def train_step(self, Tin, Ttar, lr: float, want_grad: bool = False, ctx=None, power: int = 2):
        """Loss mean(rel. error^power) of the window Tin -> Ttar and (lr > 0) one
        Adam step on the coefficients; `ctx` (same atom count) supplies the
        neighbour list and K.  With want_grad, also dL/d(nu, mut, kap, gam) as a
        (4, stages + 1) array."""
        loss = ctypes.c_float()
        g = np.empty(4 * (self.stages + 1), dtype=np.float32) if want_grad else None
        c = ctx if ctx is not None else self.ctx
        _check(self._lib.ehc_cheb_train_step(self._h, c._h, _ptr(Tin), _ptr(Ttar), ctypes.c_float(lr), int(power),
                                             ctypes.byref(loss), g.ctypes.data_as(_P) if g is not None else None),
               "ehc_cheb_train_step")
        if want_grad:
            return float(loss.value), g.reshape(4, self.stages + 1)
        return float(loss.value)

    def train_rollout(self, Tin, Ttargets, lr: float, want_grad: bool = False, ctx=None, power: int = 8):
        """Loss of len(Ttargets) windows chained from Tin against the plain
        trajectory Ttargets (a (K, N) tensor, or a list of K tensors, caller
        order) and (lr > 0) one Adam step on the coefficients."""
        import torch
        tt = torch.stack(list(Ttargets)).contiguous() if not isinstance(Ttargets, torch.Tensor) else Ttargets
        tt = tt.to(torch.float64).contiguous()
        loss = ctypes.c_float()
        g = np.empty(4 * (self.stages + 1), dtype=np.float32) if want_grad else None
        c = ctx if ctx is not None else self.ctx
        _check(self._lib.ehc_cheb_train_rollout(self._h, c._h, _ptr(Tin), _ptr(tt), int(tt.shape[0]),
                                                ctypes.c_float(lr), int(power), ctypes.byref(loss),
                                                g.ctypes.data_as(_P) if g is not None else None),
               "ehc_cheb_train_rollout")
        if want_grad:
            return float(loss.value), g.reshape(4, self.stages + 1)
        return float(loss.value)

    def predict(self, Tin, ctx=None):
        """Flux-only prediction of one window from Tin (caller order)."""
        import torch
        out = torch.empty_like(Tin)
        c = ctx if ctx is not None else self.ctx
        _check(self._lib.ehc_cheb_predict(self._h, c._h, _ptr(Tin), _ptr(out)), "ehc_cheb_predict")
        return out

    def stability(self) -> float:
        """Largest X with |P(x)| <= 1 on [0, X] for the current coefficients."""
        b = ctypes.c_double()
        _check(self._lib.ehc_cheb_stability(self._h, ctypes.byref(b)), "ehc_cheb_stability")
        return float(b.value)

    def spectrum(self, Tin=None, iters: int = 200, ctx=None) -> float:
        """tau_w K |lambda_max| of the linearised flux at Tin (or the context's
        state), by power iteration; the largest estimate bounds training's
        stability range."""
        x = ctypes.c_double()
        c = ctx if ctx is not None else self.ctx
        _check(self._lib.ehc_cheb_spectrum(self._h, c._h, _ptr(Tin) if Tin is not None else None, int(iters),
                                           ctypes.byref(x)), "ehc_cheb_spectrum")
        return float(x.value)
