/*
 * ehc.h -- C ABI of libehc: per-atom electronic heat conduction for
 * two-temperature molecular dynamics on one GB300 GPU (sm_103a).
 *
 * Method: Ullah & Ponga, "A new approach for electronic heat conduction in
 * molecular dynamics simulations" (arXiv 1810.12357), Sec. 2.  Every atom
 * carries an electronic temperature T_i; between two MD steps the library
 * advances it by explicit substeps of the master equation (Eq. HeatTransport)
 * with the pair rate of Eq. Kij, couples it to a local lattice temperature
 * (Sec. 2, T_i^lat) through the constant G, and hands the exchanged energy to
 * the atoms (Eqs. RateExchange, Motion, WorkDone, Xi).
 *
 * Conventions shared by every call:
 *  - Units: Angstrom, fs, eV, amu, K on the atom side; material constants in SI
 *    (J, W, m, K) as the paper states them; converted once in ehc_create.
 *  - Per-atom arrays the caller passes are in the caller's ("original") atom
 *    order, FP64, and live in device memory unless a name ends in _host.
 *    The library only borrows them for the duration of the call.
 *  - All GPU work is queued on the CUDA stream given to ehc_create (NULL: the
 *    legacy default stream) and is asynchronous unless a call says it syncs.
 *  - Return value: EHC_OK (0) or a negative EHC_E_* code.  Errors found on the
 *    device (theta outside [0,1], NaN, neighbour-list overflow, atoms outside a
 *    non-periodic box) are sticky in a device word and are returned by the next
 *    call that synchronises (ehc_build_neighbors, ehc_energy, ehc_sync).
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef EHC_H
#define EHC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EHC_OK 0
#define EHC_E_INVAL (-1)        /* bad argument or size */
#define EHC_E_NOMEM (-2)        /* device or host allocation failed */
#define EHC_E_CUDA (-3)         /* CUDA runtime error */
#define EHC_E_UNSTABLE (-4)     /* substep violates dt (2 n_max K + G/C_e) <= 2 */
#define EHC_E_RANGE (-5)        /* theta = T/T_max left [0,1] or became NaN, or a velocity
                                   component reached 256 A/fs (or NaN) at a build */
#define EHC_E_NBR_OVERFLOW (-6) /* an atom has more neighbours than max_neighbors (or, with
                                   skin_A > 0, more than 48 candidates within rc_A + skin_A) */
#define EHC_E_TIMEOUT (-7)      /* a bounded device wait gave up */
#define EHC_E_STATE (-8)        /* call order violated (e.g. substep before build) */
#define EHC_E_BOUNDS (-9)       /* atom outside the extent of a non-periodic axis */
#define EHC_E_INDEX (-10)       /* a gathered index outside its table (found only by
                                   the bounds-checked build, libehc_checked.so) */

/* Parameters of one system.  Paper references:
 *   Tmax_K          T^e_max of the normalisation theta = T/T_max, T_min = 0 (Sec. 2)
 *   gamma_Ce        C_e = gamma T_e (Sec. 2) [J m^-3 K^-2]; Ce_cap_kB > 0 caps C_e at
 *                   Ce_cap_kB * k_B per atomic volume
 *   kappa0, kappa_mode  kappa_e = kappa0 (mode 0) or kappa0 <T_e>/<T_lat> (mode 1, Sec. 2);
 *                   C_e and kappa_e use the system means at the start of each MD step
 *                   (per atom with ce_mode 1)
 *   dim_d, zb2_A2   d and Z b^2 of Eq. Kij: K = 2 kappa_e d / (C_e Z b^2) [1/fs]
 *   G               electron-phonon coupling of Eq. HeatTransport [W m^-3 K^-1]
 *   eps_ke_eV       atoms with own kinetic energy below this do not exchange (Eq. Xi guard)
 *   rc_A            neighbour cutoff, inclusive (Sec. 2 T_i^lat and Sec. 2.1)
 *   dt_sub_fs       electronic substep (Sec. 2.1 sub-stepping)
 *   vatom_A3        V_atom = V/N (Eq. RateExchange); <= 0 means box volume / N
 *   couple_mode     0: damping of Eq. Motion (paper); 1: Langevin friction + random
 *                   force with the same exact energy hand-over
 *   frozen          1: velocities are never changed (the lattice is a bookkeeping sink)
 *   dof_mode        0: T_lat divisor (3/2) k_B N_j (paper); 1: (3/2) k_B (N_j - 1)
 *   flux_prec       0: pair flux in FP32 on the (T - Tref)/Tmax mirror, substep state as a
 *                   float pair (about 48 bits), T kept in FP64 between calls, per-atom
 *                   exchanged energy in FP64; 1: everything in FP64
 *   Tref_K          reference temperature of the FP32 mirror
 *   laser_*         optional source of Eq. LaserIntesity (Sec. 5): absorbed fluence,
 *                   penetration length, pulse centre and standard deviation
 *   seed            Philox4x32-10 key of the Langevin random force
 *   max_neighbors   width of the neighbour table (<= 0: 32, at most 64)
 *   use_graph       1: replay substep loops from a captured CUDA graph
 *   rate_shell_n    0: every pair of the list exchanges at the rate K of Eq. Kij (paper);
 *                   n > 0: pair (i, j) at the rate K w_ij, w_ij = S2 / (n r_ij^2) with
 *                   S2 = zb2_A2 and r_ij the pair distance at the build: the weight
 *                   b^2 / r^2 renormalised so that sum_j w_j r_j^2 over an ideal shell of
 *                   n neighbours with second moment S2 stays S2 (the continuum
 *                   conductivity is unchanged; no counterpart in the paper, where K_ij
 *                   is one rate for all pairs; the weights are computed and kept in
 *                   single precision).  Weighted contexts use the general
 *                   single-precision or the FP64 substep kernel, not the row tiles
 *   ce_mode         0: C_e and kappa_e at the system means of the MD step (Sec. 2, as in the
 *                   paper); 1: LOCAL per-atom form: C_e,i = min(gamma T_i, cap), kappa_i =
 *                   kappa0 T_i / T_lat (kappa_mode 1) or kappa0, pair energy rates
 *                   (2 d / Z b^2) kappa_ij T_max f_ij with kappa_ij = (kappa_i + kappa_j) / 2;
 *                   each substep advances the atom's electron energy density U = int C_e dT
 *                   and inverts it in closed form, so sum_i U_i is conserved and the ledger's
 *                   E_e is sum_i V_atom U(T_i).  Runs on the row tiles (one series order for
 *                   each substep, from the previous substep's largest |Delta|), the general
 *                   single-precision kernel (laser source, pair weights, wide tables) and the
 *                   FP64 kernel; no border (ehc_set_border: EHC_E_STATE), batch,
 *                   network or window training (EHC_E_INVAL); ehc_cheb_step and ehc_nn_step
 *                   advance such a context with plain substeps.  The stability number is
 *                   dt (2 n_max K + G / C_min) with K = 2 d kappa0 / (gamma Z b^2 T_lat)
 *                   (times T_hi / T_c above the cap) or 2 d kappa0 / (Z b^2 C_e(T_min))
 *   pot_*           lattice forces of ehc_forces (the paper's MD runs use an EAM potential;
 *                   this library carries a pair potential for the velocity-Verlet lattice
 *                   side): Morse phi(r) = D [e^{-2 alpha (r - r0)} - 2 e^{-alpha (r - r0)}] in
 *                   shifted-force form on the neighbour list (energy and force vanish at
 *                   rc_A); pot_D_eV = 0 gives zero forces
 *   stop_*          electronic stopping (Sec. 5 cascades: a friction force on atoms above a
 *                   kinetic-energy cut, 10 eV there): in ehc_couple an atom with kinetic
 *                   energy K > stop_ecut_eV loses K (1 - e^{-2 beta dt_md}) (m dv/dt = -beta m v
 *                   over the MD step) to its own electrons, through the same exact hand-over
 *                   as A_i; stop_beta_per_fs = 0 switches it off
 *   tile_threads    threads owning atoms in the row-tile substep kernel: 0 = chosen by a
 *                   timing tuner on the first substep call of 8 or more substeps (and after
 *                   tiles grow), 256 or 128 = fixed; both give identical results
 *   tile_grid_quarters  with tile_threads fixed: the row-tile kernel's persistent grid in
 *                   quarters of its resident CTAs (2, 3 or 4; 0 = 4); with tile_threads = 0
 *                   the tuner times both widths with 4, 3 and 2 quarters (12 substeps of a
 *                   call of 16 or more) and keeps the fastest, another choice than (256, 4)
 *                   only if 3 % faster; every choice gives identical results
 *   skin_A          skin of the neighbour search (0 <= skin_A <= rc_A; 0: none): cells are
 *                   at least rc_A + skin_A wide, and a build takes the list from candidates
 *                   (the atoms within rc_A + skin_A at the last candidate build) by the
 *                   same exact integer test on the current positions, rebuilding the
 *                   candidates only when some atom moved more than skin_A / 2 since; the
 *                   list is the one the full search gives, in the same order.  A negative
 *                   value sizes the cells the same way and searches them in full every
 *                   build.  Used on grids with at least 3 cells per periodic axis, uniform
 *                   pair rates and max_neighbors <= 32; other contexts search in full.  At
 *                   most 48 candidates per atom (more: EHC_E_NBR_OVERFLOW at the build; an
 *                   FCC lattice at 300 K has about 19 within rc_A + 0.3 A for rc_A = 4 A) */
typedef struct ehc_params {
  double rc_A;
  double dt_sub_fs;
  double Tmax_K;
  double Tref_K;
  double gamma_Ce;
  double Ce_cap_kB;
  double kappa0;
  double G;
  double eps_ke_eV;
  double zb2_A2;
  double vatom_A3;
  double laser_fluence_Jm2;
  double laser_lp_A;
  double laser_t0_fs;
  double laser_sigma_fs;
  uint64_t seed;
  int32_t dim_d;
  int32_t kappa_mode;
  int32_t couple_mode;
  int32_t frozen;
  int32_t dof_mode;
  int32_t flux_prec;
  int32_t laser_on;
  int32_t max_neighbors;
  int32_t use_graph;
  int32_t tile_threads;
  int32_t rate_shell_n;
  int32_t ce_mode;
  int32_t tile_grid_quarters;
  int32_t reserved[3];
  double pot_D_eV;          /* Morse pair potential of ehc_forces (0: no forces) */
  double pot_alpha_perA;
  double pot_r0_A;
  double stop_beta_per_fs;  /* electronic stopping rate in ehc_couple (0: none) */
  double stop_ecut_eV;      /* kinetic energy above which an atom is stopped */
  double skin_A;            /* neighbour-search skin (0: none; see below) */
} ehc_params;

/* Energy ledger and diagnostics (Sec. 3.2 energy balance).  E_e is tracked
 * incrementally: E_e0 = sum_i V_atom int_0^{T_i} C_e(T) dT at ehc_set_te, then
 * each MD step adds V_atom C_e sum_i dT_i with that step's C_e.  E_lat is the
 * kinetic energy the lattice received, E_src the energy of the source term.
 * drift = (E_e + E_lat - E_src + E_res - E_e0) / max(|E_e0|, |E_e|). */
typedef struct ehc_energy_t {
  double E_e, E_lat, E_src, E_e0, drift;
  double sum_T, max_T, mean_T;
  double Te_mean_step, Tlat_step;   /* system means used for C_e, kappa_e this MD step */
  double Ce_SI, K_per_fs, stability; /* stability = dt (2 n_max K + G/C_e), must be <= 2 */
  int64_t n_stopped;                /* atoms whose kinetic energy could not pay A_i */
  int64_t md_step;
  int32_t max_count;                /* largest neighbour count */
  int32_t device_error;             /* bit set of device-side error flags */
  double E_res;                     /* energy absorbed by the fixed-temperature border
                                       (ehc_set_border), 0 without one */
} ehc_energy_t;

typedef struct ehc_ctx ehc_ctx;

/* Create a context for n_atoms atoms in an orthorhombic box [0, box_A[k]).
 * periodic[k] != 0 makes axis k periodic (box_A[k] must then exceed 2 r_c).
 * mass_amu_host: n_types masses (host memory, 1 <= n_types <= 16).
 * type_dev: per-atom type index in original order (device, int32), or NULL when
 * n_types == 1.  stream: a cudaStream_t or NULL.  Allocates all device memory
 * the context will use; no later call allocates.  *out receives the context. */
int ehc_create(const ehc_params *p, int64_t n_atoms, const double box_A[3],
               const int32_t periodic[3], const double *mass_amu_host, int32_t n_types,
               const int32_t *type_dev, void *stream, ehc_ctx **out);

/* Copy the initial electronic temperatures Te_dev [N] (original order, device)
 * into the context and reset the energy ledger (E_e0). */
int ehc_set_te(ehc_ctx *c, const double *Te_dev);

/* Per-atom depth below the irradiated surface [A] (device, original order), used
 * by the laser source of Eq. LaserIntesity.  Kept until replaced. */
int ehc_set_depth(ehc_ctx *c, const double *depth_dev);

/* Start of an MD step: bin atoms into cells, build the full neighbour list
 * (all j != i with |x_j - x_i| <= r_c on a 2^-20 A fixed-point grid, minimum
 * image on periodic axes; Sec. 2), compute the local lattice temperature of
 * every atom from its neighbours' velocities (Sec. 2, T_i^lat, centre-of-mass
 * velocity removed), the system means <T_e> and T_lat = K/((3/2) k_B N), and from
 * them C_e, kappa_e and K of Eq. Kij for this step.  x_dev, v_dev: [N,3].
 * Synchronises the stream once (reads back a few scalars). */
int ehc_build_neighbors(ehc_ctx *c, const double *x_dev, const double *v_dev);

/* n_sub explicit Euler substeps of Eq. HeatTransport (all atoms read the same
 * snapshot), starting at time t_fs (used by the laser source).  Returns
 * EHC_E_UNSTABLE without launching if dt (2 n_max K + G/C_e) > 2.  Allocates
 * nothing; asynchronous. */
int ehc_substep(ehc_ctx *c, int32_t n_sub, double t_fs);

/* End of an MD step: hand the energy each atom's electrons gave up during the
 * substeps to its velocity (Eqs. RateExchange, WorkDone, Xi), in place on v_dev
 * [N,3].  dt_md_fs is the MD step (Langevin friction and noise amplitude). */
int ehc_couple(ehc_ctx *c, double *v_dev, double dt_md_fs);

/* Fixed-temperature electron border (a Dirichlet condition on T_e, as the 300 K
 * border shell of the paper's cascade runs, Sec. 5; no other counterpart in the
 * paper).  Tfix_dev [N] (caller order, device, copied): atom i with a finite
 * Tfix_dev[i] is an electron reservoir held at that temperature (0..Tmax_K, else
 * EHC_E_RANGE at the build); NaN marks a free atom; NULL removes the border.
 * Takes effect at the next ehc_build_neighbors.  Every substep is taken for all
 * atoms (a border atom exchanges pair fluxes and coupling energy at its fixed
 * T), then border atoms are put back to their temperature; what they would have
 * gained, times V_atom C_e, is the reservoir energy E_res of ehc_energy, which
 * closes the ledger.  The build sets border atoms to their Tfix and charges a
 * difference to the reservoir (set T_e of border atoms to Tfix in ehc_set_te to
 * avoid one).  The
 * first call allocates 17 bytes per atom.  With a border, ehc_cheb_step and
 * ehc_nn_step advance by plain substeps (counted as fallbacks) and ehc_save
 * returns EHC_E_STATE. */
int ehc_set_border(ehc_ctx *c, const double *Tfix_dev);

/* Free flight x += v dt, wrapped into the box on periodic axes: the position
 * update of the velocity-Verlet step (and the whole lattice step when no
 * interatomic forces are used). */
int ehc_drift(ehc_ctx *c, double *x_dev, const double *v_dev, double dt_fs);

/* Interatomic forces F_i of Eq. Motion from the shifted-force Morse potential
 * (ehc_params.pot_*) at the positions of the last ehc_build_neighbors, over its
 * neighbour list (pairs with r <= rc_A): F_dev [N,3] eV/A, caller order, written
 * (device, caller-owned).  Pair terms in single precision on the exact integer
 * displacements of the quantised positions, sums per atom in single precision,
 * the potential energy summed in FP64 into *epot_host [eV] when epot_host is not
 * NULL (then the call synchronises).  EHC_E_STATE before the first build. */
int ehc_forces(ehc_ctx *c, double *F_dev, double *epot_host);

/* Velocity-Verlet kick of Eq. Motion's interatomic part, v_i += dt F_i / m_i
 * (caller order, per-type masses, F in eV/A, v in A/fs; v_dev [N,3] updated in
 * place, F_dev [N,3] read; both device, caller-owned): called with dt = half the
 * MD step before the drift and after the forces of the new positions (the
 * damping/friction part of Eq. Motion is ehc_couple's).  Asynchronous. */
int ehc_kick(ehc_ctx *c, double *v_dev, const double *F_dev, double dt_fs);

/* Ghost exchange of a domain-decomposed run (one context per domain: its owned
 * atoms plus the ghost atoms their neighbour rows reach; the paper's MPI fix
 * exchanged the ghosts' electronic temperatures before every substep, Sec. 2.1).
 * ehc_get_te_at writes the current T_e of the caller-order atoms idx_dev[0..m)
 * (int32, device) to out_dev[0..m) (FP64, device); ehc_set_te_at overwrites
 * them with vals_dev[0..m) between substep calls, the single-precision state
 * included (the next substep then evaluates the full series everywhere).
 * Indices outside [0, n) are skipped and reported as EHC_E_INDEX by the next
 * synchronising call.  EHC_E_STATE before ehc_set_te.  Asynchronous.
 * The context's own ledger (ehc_energy) is left alone by ehc_set_te_at: in a
 * domain context it counts the ghosts' electronic energy, which the exchange
 * overwrites, so a domain's drift is not a conservation check.  The conserved
 * ledger of a decomposed run is the all-reduced one: E_e changes with
 * V_atom C_e sum T over the owned atoms (ehc_sums_at), the exchanged energies
 * with the owned atoms' hand-over. */
int ehc_get_te_at(ehc_ctx *c, const int32_t *idx_dev, int64_t m, double *out_dev);
int ehc_set_te_at(ehc_ctx *c, const int32_t *idx_dev, int64_t m, const double *vals_dev);

/* Sums over the caller-order atoms idx_dev[0..m) of this context for the
 * all-reduce of a domain-decomposed run: sums_host[0] = sum T_e [K] (current),
 * sums_host[1] = sum (1/2) m |v|^2 [eV] with the velocities of the last build
 * (the sums the build's system means are made of).  Deterministic (fixed grid).
 * Synchronises; EHC_E_INDEX if an index is outside [0, n), EHC_E_STATE before
 * the first build. */
int ehc_sums_at(ehc_ctx *c, const int32_t *idx_dev, int64_t m, double *sums_host);

/* System means of the MD step (Sec. 2: mean electronic and classical lattice
 * temperature) in place of the ones the last ehc_build_neighbors computed from
 * this context's atoms: for a domain of a decomposed system, whose means are the
 * all-reduced sums over the owned atoms of every domain divided by the total
 * count.  Recomputes C_e, kappa_e, K and the stability number for the step's
 * substeps and hand-over.  EHC_E_STATE before the first build. */
int ehc_set_step_means(ehc_ctx *c, double Te_mean, double Tlat);

/* Key of the Langevin hand-over's random stream (the random-force coupling the
 * paper cites beside Eqs. Motion and Xi; Philox4x32-10 counter = (atom id, MD
 * step), key = seed).  By default atom i of the caller order draws with id i and
 * the MD step counts this context's ehc_couple calls from 0.  A domain of a
 * decomposed system renumbers its atoms and is a new context every MD step, so
 * it sets ids_dev[0..n) (int64, device, caller order; copied, the caller keeps
 * ownership) to the atoms' global ids and md_step to the system's MD step: its
 * atoms then draw the numbers the undivided run draws.  ids_dev null returns to
 * the caller index (md_step is set either way).  The ids are not checked for
 * uniqueness (equal ids draw equal numbers) and are not part of a checkpoint.
 * The first call with ids allocates n int64 on the device (EHC_E_NOMEM);
 * EHC_E_INVAL for md_step < 0.  Asynchronous on the context stream. */
int ehc_set_rng_ids(ehc_ctx *c, const int64_t *ids_dev, int64_t md_step);

/* Failure-detection probe of the bounded device waits (no counterpart in the
 * paper): one block waits, with the mbarrier poll loop of the row-tile kernels
 * and a budget of `polls` polls, on a phase that completes (complete != 0) or
 * that nothing completes (complete = 0).  Returns EHC_E_TIMEOUT when the wait
 * ran out, EHC_OK otherwise; the result travels in a word of its own, so the
 * context's error state is untouched and the context stays usable.
 * Synchronises.  EHC_E_INVAL for polls = 0. */
int ehc_probe_wait(ehc_ctx *c, uint32_t polls, int32_t complete);

/* Largest speed max_i |v_i| [A/fs] of v_dev [N,3] into *vmax_host, for a variable
 * MD step (the cascade runs of Sec. 5 cap the displacement per step).  Synchronises. */
int ehc_max_speed(ehc_ctx *c, const double *v_dev, double *vmax_host);

/* One whole MD step with HOST buffers: copies x_host, v_host [N,3] to the
 * device, runs build, n_sub substeps from t_fs, couple and drift, and copies
 * x, v and the electronic temperatures back (Te_host_out [N]).  The velocity
 * upload overlaps the binning and neighbour search, its download the drift (on
 * a second stream of the context).  Host buffers should be page-locked for full
 * copy speed.  Synchronises. */
int ehc_md_step_host(ehc_ctx *c, double *x_host, double *v_host, int32_t n_sub,
                     double t_fs, double dt_md_fs, double *Te_host_out);

/* Energy ledger and diagnostics; synchronises and returns any sticky device
 * error as its EHC_E_* code (the ledger is filled in either way). */
int ehc_energy(ehc_ctx *c, ehc_energy_t *out);

/* Wait for queued work; return a sticky device error if one was raised. */
int ehc_sync(ehc_ctx *c);

/* Electronic temperatures [N] (original order) into Te_dev_out (device). */
int ehc_get_te(ehc_ctx *c, double *Te_dev_out);

/* Local lattice temperatures of the current MD step [N] (original order, device);
 * atoms below the kinetic-energy guard are reported as -1. */
int ehc_get_lattice_temperature(ehc_ctx *c, double *Tl_dev_out);

/* Current neighbour list in canonical form: rows in original atom order, each
 * row's original ids ascending.  rowptr_host [N+1]; col_host has room for cap
 * entries.  Returns EHC_E_INVAL if cap is too small.  Synchronises. */
int ehc_export_neighbors(ehc_ctx *c, int64_t *rowptr_host, int32_t *col_host, int64_t cap);

/* Three standard normals per listed atom from the Philox4x32-10 stream the
 * Langevin hand-over uses: counter (id, md_step), key seed; out_dev [n,3]. */
int ehc_philox_normals(const int64_t *ids_dev, int64_t n, uint64_t md_step, uint64_t seed,
                       double *out_dev, void *stream);

/* Checkpoint: electronic temperatures, pending exchange energies, ledger,
 * step counter and Philox key to a file; ehc_load restores them into a context
 * created with the same parameters and atom count. */
int ehc_save(ehc_ctx *c, const char *path);
int ehc_load(ehc_ctx *c, const char *path);

/* Electronic energy of a set of temperatures without allocating anything: the
 * paper has no counterpart; this serves callers that cannot call cudaMalloc at
 * the time they need the number (an application whose device memory pool is
 * fixed at start-up, a plugin that may not touch its host code's allocator, a
 * loop that must not take the allocator's locks).  Te_dev [n] (device, any order); writes to
 * out_dev (device, 3 doubles): sum of T [K], max T [K] and
 * sum_i V_atom int_0^{T_i} C_e dT [eV] with C_e = min(gamma_Ce T, Ce_cap_kB k_B / V_atom)
 * (Ce_cap_kB <= 0: no cap) -- the E_e0 that ehc_set_te computes.  Asynchronous on
 * `stream`.  Scratch: a fixed 128 KB device array in the library, held by every
 * GPU that loads it until the process exits; n may not exceed 16,777,216
 * (EHC_E_INVAL beyond).  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture; that address is cached per device, so do not
 * use the entry point across a cudaDeviceReset.  All calls share the array and
 * every call overwrites the part it uses, so calls that overlap on the GPU
 * (different streams, or host threads) race; serialise them.  A NaN among the
 * temperatures makes max T NaN. */
int ehc_electron_energy_noalloc(const double *Te_dev, int64_t n, double gamma_Ce, double Ce_cap_kB,
                                double vatom_A3, double *out_dev, void *stream);

void ehc_destroy(ehc_ctx *c);
const char *ehc_strerror(int code);

/* ---- Learned window propagator ------------------------------------------------
 * A small message-passing network over the context's neighbour list stands in
 * for n_window explicit substeps of Eq. HeatTransport (pair-flux part); the
 * coupling term of the window is applied in closed form.  Two layers of hidden
 * width H (8 or 16), every pair term odd under i <-> j (pair fluxes conserve
 * sum_i T_i).  With delta = (T - Tref)/Tmax, D = (delta_j - delta_i)/sigma,
 * q = D^2/(1+D^2), s = theta_i + theta_j:
 *   h_i = sum_j D relu(W1 [q, s] + b1),
 *   phi_ij = D (c0 + w . relu(W2 [q, s] + b2)) + u . (h_j - h_i),
 *   T^_i = T_i + sigma Tmax (n_window dt K) sum_j phi_ij.
 * Parameters (8H + 1 floats): [W1 (H x 2) | b1 | W2 (H x 2) | b2 | w | u | c0];
 * BF16 weights and hidden vectors in the forward, FP32 arithmetic and
 * accumulation, FP32 master weights and Adam for training.  The network is
 * bound to the atom count of the context it was created with; single-precision
 * flux, no laser source. */
typedef struct ehc_nn ehc_nn;
int ehc_nn_create(ehc_ctx *c, int32_t hidden, int32_t n_window, double sigma, ehc_nn **out);
int ehc_nn_set_params(ehc_nn *nn, ehc_ctx *c, const float *params_host);
int ehc_nn_get_params(ehc_nn *nn, ehc_ctx *c, float *params_host);
/* One training step on a window: Tin_dev -> Ttar_dev (caller order, device;
 * the target is the state after n_window plain substeps without coupling) on the
 * context's current neighbour list and K.  Loss mean(((T^ - T*)/(sigma Tmax))^2)
 * to *loss_host; the gradient (8H + 1) to grad_host if not NULL; an Adam step of
 * rate lr if lr > 0.  Synchronises. */
int ehc_nn_train_step(ehc_nn *nn, ehc_ctx *c, const double *Tin_dev, const double *Ttar_dev, float lr,
                      float *loss_host, float *grad_host);
/* Flux-only prediction of one window from Tin_dev into Tout_dev (caller order). */
int ehc_nn_predict(ehc_nn *nn, ehc_ctx *c, const double *Tin_dev, double *Tout_dev);
/* Advance the context by one window: predict, apply the window's coupling, and
 * form the a-posteriori residual rho = max_i |T^_i - T_i - tau_w (R(T)_i + R(T^)_i)/2|
 * / max(1 K, 1e-3 T_i) with R the right-hand side of Eq. HeatTransport and tau_w the
 * window length.  rho <= tau: the prediction is kept (and its coupling energy
 * handed to the lattice ledger); otherwise the window is redone with n_window
 * plain substeps (*fell_back = 1).  Synchronises once. */
int ehc_nn_step(ehc_nn *nn, ehc_ctx *c, double tau, double t_fs, int32_t *fell_back, double *rho_out);
void ehc_nn_destroy(ehc_nn *nn);

/* ---- Chebyshev window propagator ---------------------------------------------
 * A window of n_window explicit substeps of Eq. HeatTransport is advanced with
 * `stages` evaluations of the pair flux instead of n_window: the damped
 * Chebyshev recurrences (Runge-Kutta-Chebyshev family, first or second order;
 * no counterpart in the paper, which integrates with plain explicit substeps).
 * With theta = T / Tmax, tau_w = n_window dt, F_i = sum_j f(theta_i, theta_j),
 * w0 = 1 + damping / s^2 and T_j the Chebyshev polynomials (all at w0):
 *   Y_0 = theta,  Y_1 = Y_0 + mut_1 tau_w K F(Y_0),
 *   Y_j = Y_{j-1} + nu_j (Y_{j-2} - Y_{j-1}) + kap_j (Y_0 - Y_{j-1})
 *         + mut_j tau_w K F(Y_{j-1}) + gam_j tau_w K F(Y_0),   j = 2..s.
 * order 1: w1 = T_s / T_s', b_j = 1 / T_j, mut_1 = w1 / w0, nu_j = -b_j / b_{j-2},
 *   mut_j = 2 w1 b_j / b_{j-1}, kap = gam = 0; a linear mode of rate lambda is
 *   multiplied by T_s(w0 - w1 tau_w lambda) / T_s(w0), stable while tau_w lambda
 *   <= (1 + w0) / w1, about (2 - 4 damping / 3) s^2.
 * order 2: w1 = T_s' / T_s'', b_j = T_j'' / T_j'^2 (b_0 = b_1 = b_2),
 *   a_j = 1 - b_j T_j, mut_1 = b_1 w1, mu_j = 2 b_j w0 / b_{j-1}, nu_j = -b_j / b_{j-2},
 *   mut_j = 2 b_j w1 / b_{j-1}, kap_j = 1 - mu_j - nu_j, gam_j = -a_{j-1} mut_j;
 *   the multiplier a_s + b_s T_s(w0 - w1 tau_w lambda) agrees with exp(-tau_w lambda)
 *   to second order; stable to about 0.65 s^2 (damping 2/13).
 * Every stage keeps sum_i T_i.  The coupling of the window is applied after
 * the stages as in ehc_nn_step, and so are the residual test and the fallback
 * to plain substeps.  Stages run in FP32 on the row-tile path (values
 * (T - Tref)/Tmax); contexts without it always fall back.  Single-precision
 * flux, no laser source; bound to the context's atom count. */
typedef struct ehc_cheb ehc_cheb;
/* n_window >= 1, 2 <= stages <= 32, order 1 or 2, 0 <= damping <= 10
 * (EHC_E_INVAL otherwise). */
int ehc_cheb_create(ehc_ctx *c, int32_t n_window, int32_t stages, int32_t order, double damping,
                    ehc_cheb **out);
/* nu, mut and (if not NULL) kap, gam for j = 0..stages into host arrays of
 * stages + 1 doubles (index 0 unused). */
int ehc_cheb_coefficients(const ehc_cheb *w, double *nu_host, double *mut_host, double *kap_host,
                          double *gam_host);
/* Advance the context by one window (see ehc_nn_step for rho, tau and the
 * fallback).  Synchronises once. */
int ehc_cheb_step(ehc_cheb *w, ehc_ctx *c, double tau, double t_fs, int32_t *fell_back, double *rho_out);
/* windows advanced and windows redone by plain substeps since creation */
int ehc_cheb_stats(const ehc_cheb *w, int64_t *windows, int64_t *fallbacks);

/* ---- trained windows -----------------------------------------------------------
 * The stage coefficients nu, mut, kap, gam (j = 1..s) are free parameters that
 * can be set and trained on windows of the plain method, so that s stages
 * reproduce n_window explicit substeps of Eq. HeatTransport better than the
 * damped Chebyshev values they start from (a learned propagator: a message-
 * passing network of s layers whose message is the paper's pair flux and whose
 * layer weights are learned; no counterpart in the paper).  In the form of the
 * stages on the window's change z_j = Y_j - Y_0 (a_j = mut_j tau_w K,
 * g_j = gam_j tau_w K):
 *   z_1 = a_1 F(Y_0),
 *   z_j = z_{j-1} + nu_j (z_{j-2} - z_{j-1}) - kap_j z_{j-1} + a_j F(Y_{j-1}) + g_j F(Y_0).
 * Any coefficients keep sum_i T_i (every stage adds pair fluxes only). */
/* Replace the coefficients (host arrays of stages + 1 doubles, index 0 unused;
 * nu_1, kap_1 and gam_1 are ignored: stage 1 uses mut_1 only).  They become the
 * base of training: Adam works on relative changes d, c = base (1 + d), so a
 * coefficient set to 0 stays 0.  Resets the optimiser.  EHC_E_INVAL for
 * non-finite values or |c| > 1e6.  Synchronises. */
int ehc_cheb_set_coefficients(ehc_cheb *w, ehc_ctx *c, const double *nu_host, const double *mut_host,
                              const double *kap_host, const double *gam_host);
/* One training step on one window: Tin_dev -> Ttar_dev (caller order, device; the
 * target is the state after n_window plain substeps with the coupling off) on
 * the context's neighbour list and K.  Loss mean_i ((T^_i - T*_i) / Tin_i)^p,
 * p = loss_power (2, 4 or 8; the higher powers weigh the worst atoms), of the
 * s stages' prediction T^ to *loss_host; dL/d(nu, mut, kap, gam) to grad_host
 * (4 (stages + 1) floats: the four sets one after another, index j within each)
 * if not NULL.  If lr > 0, one Adam step of rate lr on the relative changes;
 * mut and gam are then rescaled so that P'(0) = -1 for the window's linear
 * stability polynomial P (slow modes decay at the plain rate), and the step is
 * halved (up to 20 times, else not taken) until |P(x)| <= 1 + 1e-6 on a grid of
 * 16384 points of 0 < x <= X_r, X_r = 1.1 x the largest ehc_cheb_spectrum
 * estimate so far, or 1.1 n_window s_c without one (s_c the context's
 * per-substep stability number, a bound of dt lambda_max).  Training must start
 * from coefficients that meet this (EHC_E_UNSTABLE otherwise, nothing changed).
 * Forward and backward run on the GPU (one thread per atom on the neighbour
 * list, single precision, FP64 reductions); the first call allocates
 * (1 + 3 stages) floats per atom.  Synchronises. */
int ehc_cheb_train_step(ehc_cheb *w, ehc_ctx *c, const double *Tin_dev, const double *Ttar_dev, float lr,
                        int32_t loss_power, float *loss_host, float *grad_host);
/* Estimate x = tau_w K |lambda_max| of the linearised pair flux at the state
 * Tin_dev (caller order, device) or, if NULL, at the context's T, by `iters`
 * (1..100000) power iterations with the transposed Jacobian; to *x_out.  The
 * largest estimate so far bounds the stability range of training.  The
 * iteration approaches |lambda_max| from below. */
int ehc_cheb_spectrum(ehc_cheb *w, ehc_ctx *c, const double *Tin_dev, int32_t iters, double *x_out);
/* One training step on a rollout: n_win (1..64) windows chained from Tin_dev,
 * each started from the previous one's end, against the plain method's states
 * after each window, Ttar_dev [n_win][N] (caller order, device, coupling off).
 * Loss sum_w mean_i ((T^_w,i - T*_w,i) / T*_w,i)^p, p = loss_power (2, 4, 8); its
 * gradient by the adjoint through the chain (GPU kernels: the stage sweep of
 * each window in reverse, the window-start adjoint passed back); gradient and
 * Adam step as in ehc_cheb_train_step (same stability constraint, same
 * EHC_E_UNSTABLE).  The first call with a given n_win allocates
 * (n_win + 1 + 2 n_win stages + 5) floats and n_win doubles per atom.
 * Synchronises. */
int ehc_cheb_train_rollout(ehc_cheb *w, ehc_ctx *c, const double *Tin_dev, const double *Ttar_dev, int32_t n_win,
                           float lr, int32_t loss_power, float *loss_host, float *grad_host);
/* The stages' flux-only prediction of one window from Tin_dev into Tout_dev
 * (caller order, device), with the training kernels.  Training, prediction and
 * the spectrum estimate take uniform pair rates only (EHC_E_INVAL with
 * rate_shell_n > 0); windows of weighted contexts run as plain substeps. */
int ehc_cheb_predict(ehc_cheb *w, ehc_ctx *c, const double *Tin_dev, double *Tout_dev);
/* Largest X such that |P(x)| <= 1 + 1e-5 on [0, X] for the current coefficients
 * (the window is stable for modes with tau_w lambda <= X), scanned on 200000
 * points of [0, 2.05 stages^2]; host computation. */
int ehc_cheb_stability(const ehc_cheb *w, double *beta);
void ehc_cheb_destroy(ehc_cheb *w);

/* ---- Learned corrector of the window propagator ---------------------------------
 * A two-layer message-passing network over the context's neighbour list (node
 * width 64) adds a learned pair flux to a window's result Y, so that the window
 * follows n_w plain substeps of Eq. HeatTransport more closely (the paper has no
 * network; it stands in for substeps of Eq. HeatTransport, Sec. 2.1).  With
 * delta = (Y - Tref)/Tmax, D_ij = (delta_j - delta_i)/sigma, q_ij = D^2/(1 + D^2),
 * rho_ij = r_ij / r_c, node features f_i = [Y_i/1e4, T_l,i/1e3 (0 below the
 * kinetic-energy guard), z_i/18] (z_i the neighbour count) and <.> the mean over
 * the atom's row:
 *   in_i = [f_i, <f_j>, <q>, <q^2>, <rho>, <q rho>, 1, 0 x 5]                  (16)
 *   h1 = relu(W1 in + b1), h2 = relu(W2 h1 + b2), u = W3 h2                 (64, 64, 16)
 *   g_ij = w4 . relu(u_i + u_j + P [q_ij, rho_ij] + b4)                    (symmetric)
 *   Y^_i = Y_i + kappa sum_j (Y_j - Y_i) g_ij,  kappa = n_w dt_sub K in a window.
 * Every pair term is odd under i <-> j, so sum_i Y_i is kept.  The node MLP runs
 * on the tensor cores with BF16 weights and activations and FP32 accumulation;
 * the edge MLP in FP32 from BF16 weights.  Parameters (6336 floats): [W1 (64 x 16)
 * | b1 (64) | W2 (64 x 64) | b2 (64) | W3 (16 x 64) | P (16 x 2) | b4 (16) | w4 (16)],
 * row-major (out x in); FP32 master weights and Adam for training.  Zero weights
 * (as created) make the identity.  The corrector is bound to the atom count of
 * the context it was created with; single-precision flux and uniform pair rates
 * only (EHC_E_INVAL otherwise). */
typedef struct ehc_gnn ehc_gnn;
int ehc_gnn_create(ehc_ctx *c, double sigma, ehc_gnn **out);
/* set (resets Adam) or read the FP32 parameters [6336] (host); synchronise */
int ehc_gnn_set_params(ehc_gnn *g, ehc_ctx *c, const float *params_host);
int ehc_gnn_get_params(ehc_gnn *g, ehc_ctx *c, float *params_host);
/* Y^ of Y_dev into Yhat_dev (caller order, device) on the context's current
 * neighbour list and lattice temperatures; the correction Y^ - Y into dY_dev if
 * not NULL.  Asynchronous; EHC_E_STATE before the first build. */
int ehc_gnn_apply(ehc_gnn *g, ehc_ctx *c, double kappa, const double *Y_dev, double *Yhat_dev, double *dY_dev);
/* One training step on a window: Y_dev the propagator's result, Tstar_dev the
 * plain substeps' (caller order, device).  Loss mean(((Y^ - T*)/T*)^2) to
 * *loss_host, its gradient [6336] to grad_host if not NULL, an Adam step of rate
 * lr if lr > 0.  Synchronises. */
int ehc_gnn_train_step(ehc_gnn *g, ehc_ctx *c, double kappa, const double *Y_dev, const double *Tstar_dev,
                       float lr, float *loss_host, float *grad_host);
/* Apply g (or no corrector: NULL) to the result of every window ehc_cheb_step
 * takes with w, before its residual test; g stays owned by the caller and must
 * outlive its use by w. */
int ehc_cheb_set_corrector(ehc_cheb *w, ehc_gnn *g);

/* The row-tile kernel's width (threads owning atoms: 256 or 128) and persistent
 * grid (quarters of its resident CTAs) this context runs with: the tuner's choice
 * after the first substep call of 16 or more substeps, or the fixed values of
 * ehc_params; (0, 0) before either.  A caller can keep the choice for later
 * contexts of the same shape (the Python binding caches it per GPU and shape). */
int ehc_tuning(ehc_ctx *c, int32_t *tile_threads, int32_t *grid_quarters);
void ehc_gnn_destroy(ehc_gnn *g);

/* ---- Batched replicas --------------------------------------------------------
 * Independent systems (e.g. repeated cascades of different sizes, Sec. 4) that
 * share one parameter set are advanced together: each replica keeps its own
 * neighbour list, per-step C_e / kappa_e / K and energy ledger exactly as a
 * single context would, and the substeps of all replicas run as one launch per
 * substep over a work list of (replica, row) tiles, replayed from a CUDA graph.
 * Per-atom arrays are the replicas' arrays concatenated in replica order
 * (positions and velocities [sum n, 3]); ehc_batch_size gives the offsets.
 * Single-precision flux only (flux_prec 0), no laser source, one atom type.
 * The results of a replica are those a single context gives for it. */
typedef struct ehc_batch ehc_batch;

/* n_rep replicas with n_atoms_host[r] atoms in boxes boxes_host[3 r .. 3 r + 2]
 * (host memory), all with the same periodic flags and the one atom mass. */
int ehc_batch_create(const ehc_params *p, int32_t n_rep, const int64_t *n_atoms_host,
                     const double *boxes_host, const int32_t periodic[3], const double *mass_amu_host,
                     void *stream, ehc_batch **out);
/* total atom count and the first atom of every replica (offsets_host [n_rep], may be NULL) */
int ehc_batch_size(const ehc_batch *b, int64_t *n_total, int64_t *offsets_host);
int ehc_batch_set_te(ehc_batch *b, const double *Te_dev);
/* one neighbour build for every replica; synchronises the stream once */
int ehc_batch_build_neighbors(ehc_batch *b, const double *x_dev, const double *v_dev);
int ehc_batch_substep(ehc_batch *b, int32_t n_sub, double t_fs);
int ehc_batch_couple(ehc_batch *b, double *v_dev, double dt_md_fs);
int ehc_batch_drift(ehc_batch *b, double *x_dev, const double *v_dev, double dt_fs);
int ehc_batch_get_te(ehc_batch *b, double *Te_dev_out);
/* ledger of replica r */
int ehc_batch_energy(ehc_batch *b, int32_t r, ehc_energy_t *out);
/* the batch's row-tile width and grid share, as ehc_tuning (ehc_params of the
 * batch: tile_threads, tile_grid_quarters) */
int ehc_batch_tuning(ehc_batch *b, int32_t *tile_threads, int32_t *grid_quarters);
void ehc_batch_destroy(ehc_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* EHC_H */
