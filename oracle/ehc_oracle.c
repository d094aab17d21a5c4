/*
 * ehc_oracle.c -- plain, slow FP64 CPU oracle of the l2T-MD electronic
 * heat-conduction step (Ullah & Ponga, arXiv 1810.12357).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant with the CUDA library; it is written from the paper's equations.
 *
 * Compiled with -O2 -fno-fast-math -ffp-contract=off, so every expression is
 * evaluated as written in IEEE double precision.  Loops over atoms may run in
 * parallel (OpenMP); each atom's sum is taken over its neighbour row in
 * ascending original-id order, so results do not depend on the thread count.
 *
 * Units: Angstrom, fs, eV, amu, K.  Positions are mapped to a 2^-20 Angstrom
 * fixed-point grid so that the neighbour test is exact integer arithmetic.
 *
 * Parity status of each function: see the pins listed beside it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 */
static const double O_KB = 8.617333262e-5;          /* eV / K */
static const double O_AMU = 1.66053906660e-27;      /* kg */
static const double O_EV = 1.602176634e-19;         /* J */

static double o_mvv_ev(void) { return O_AMU * 1.0e10 / O_EV; } /* amu*(A/fs)^2 in eV */

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Fixed-point positions.  Neighbour selection "x_j - x_i <= r_c" (Sec. 2,
 * lattice-temperature definition) evaluated exactly on integers.
 * q = round-half-even(x * 2^20); periodic axes wrapped into [0, Lq).
 * Pins: brute-force vs cell search; 18 neighbours per atom in perfect FCC Cu. */
int oracle_quantize(int64_t n, const double *x, const double *box, const int32_t *periodic,
                    int32_t *q, int64_t *Lq_out) {
  int64_t Lq[3];
  for (int k = 0; k < 3; ++k) {
    Lq[k] = llrint(box[k] * 1048576.0);
    Lq_out[k] = Lq[k];
    if (Lq[k] <= 0 || Lq[k] >= 2147483647LL) return -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) {
      int64_t v = llrint(x[3 * i + k] * 1048576.0);
      if (periodic[k]) {
        v %= Lq[k];
        if (v < 0) v += Lq[k];
      } else if (v < 0 || v >= Lq[k]) {
        return -2; /* atoms must lie inside non-periodic extents */
      }
      q[3 * i + k] = (int32_t)v;
    }
  }
  return 0;
}

/* Minimum-image displacement on the integer grid; a displacement of exactly
 * half the box keeps its sign. */
static int64_t o_disp(int64_t d, int64_t L, int per) {
  if (per) {
    if (2 * d > L) d -= L;
    else if (2 * d < -L) d += L;
  }
  return d;
}

static int o_within(const int32_t *qi, const int32_t *qj, const int64_t *Lq, const int32_t *per,
                    int64_t rcq) {
  int64_t s = 0;
  for (int k = 0; k < 3; ++k) {
    int64_t d = o_disp((int64_t)qj[k] - (int64_t)qi[k], Lq[k], per[k]);
    if (d > rcq || d < -rcq) return 0;
    s += d * d;
  }
  return s <= rcq * rcq;
}

/* O(N^2) reference search: row i lists every j != i with |x_j - x_i| <= r_c,
 * ascending j.  Returns the number of entries, or -1 if cap is exceeded. */
int64_t oracle_neighbors_brute(int64_t n, const int32_t *q, const int64_t *Lq,
                               const int32_t *periodic, int64_t rcq, int64_t *rowptr,
                               int32_t *col, int64_t cap) {
  int64_t nnz = 0;
  rowptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      if (o_within(q + 3 * i, q + 3 * j, Lq, periodic, rcq)) {
        if (nnz >= cap) return -1;
        col[nnz++] = (int32_t)j;
      }
    }
    rowptr[i + 1] = nnz;
  }
  return nnz;
}

static int o_cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Same list by a linked cell search: cells of width >= r_c, each atom looks at
 * the (deduplicated) 3x3x3 block of cells around its own.  Rows are sorted
 * ascending by original id.  Two passes: counts, then fill. */
int64_t oracle_neighbors_cells(int64_t n, const int32_t *q, const int64_t *Lq,
                               const int32_t *periodic, int64_t rcq, int64_t *rowptr,
                               int32_t *col, int64_t cap) {
  int64_t nc[3];
  for (int k = 0; k < 3; ++k) {
    nc[k] = Lq[k] / rcq;
    if (nc[k] < 1) nc[k] = 1;
    if (nc[k] > 1024) nc[k] = 1024;
  }
  int64_t ncell = nc[0] * nc[1] * nc[2];
  int64_t *head = (int64_t *)malloc(sizeof(int64_t) * ncell);
  int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  int64_t *cellof = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  if (!head || !next || !cellof) { free(head); free(next); free(cellof); return -2; }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  /* insert in descending id so every cell chain is ascending */
  for (int64_t i = n - 1; i >= 0; --i) {
    int64_t c3[3];
    for (int k = 0; k < 3; ++k) {
      int64_t c = ((int64_t)q[3 * i + k] * nc[k]) / Lq[k];
      if (c >= nc[k]) c = nc[k] - 1;
      c3[k] = c;
    }
    int64_t c = c3[0] + nc[0] * (c3[1] + nc[1] * c3[2]);
    cellof[i] = c;
    next[i] = head[c];
    head[c] = i;
  }
  int64_t *cnt = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int64_t overflow = 0;
  for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : overflow)
    for (int64_t i = 0; i < n; ++i) {
      int64_t ci[3];
      int64_t c = cellof[i];
      ci[0] = c % nc[0];
      ci[1] = (c / nc[0]) % nc[1];
      ci[2] = c / (nc[0] * nc[1]);
      /* candidate cell offsets per axis, without repeats */
      int64_t off[3][3];
      int noff[3];
      for (int k = 0; k < 3; ++k) {
        noff[k] = 0;
        for (int64_t d = -1; d <= 1; ++d) {
          int64_t cc = ci[k] + d;
          if (periodic[k]) {
            cc = ((cc % nc[k]) + nc[k]) % nc[k];
          } else if (cc < 0 || cc >= nc[k]) {
            continue;
          }
          int dup = 0;
          for (int m = 0; m < noff[k]; ++m) dup |= (off[k][m] == cc);
          if (!dup) off[k][noff[k]++] = cc;
        }
      }
      int64_t m = 0;
      int64_t base = pass ? rowptr[i] : 0;
      for (int a = 0; a < noff[2]; ++a)
        for (int b = 0; b < noff[1]; ++b)
          for (int d = 0; d < noff[0]; ++d) {
            int64_t cell = off[0][d] + nc[0] * (off[1][b] + nc[1] * off[2][a]);
            for (int64_t j = head[cell]; j >= 0; j = next[j]) {
              if (j == i) continue;
              if (o_within(q + 3 * i, q + 3 * j, Lq, periodic, rcq)) {
                if (pass) {
                  if (base + m < cap) col[base + m] = (int32_t)j;
                  else overflow += 1;
                }
                ++m;
              }
            }
          }
      if (!pass) cnt[i] = m;
      else if (base + m <= cap) qsort(col + base, (size_t)m, sizeof(int32_t), o_cmp_i32);
    }
    if (!pass) {
      rowptr[0] = 0;
      for (int64_t i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + cnt[i];
    }
  }
  free(head); free(next); free(cellof); free(cnt);
  if (overflow || rowptr[n] > cap) return -1;
  return rowptr[n];
}

/* ------------------------------------------------------------------------ */
/* Local lattice temperature (Sec. 2, T_i^lat definition): over the set S of
 * atom i and its neighbours within r_c, with the centre-of-mass velocity of S
 * removed, T_i = sum_S (1/2) m |v - v_com|^2 / ((3/2) k_B N_j), N_j = |S|.
 * dof_mode 1 divides by (3/2) k_B (N_j - 1) instead.
 * Also returns each atom's own raw kinetic energy K_i = (1/2) m v_i.v_i [eV]
 * (Eq. Xi), used by the epsilon guard.
 * Pins: a uniform-velocity set gives exactly 0; a two-atom closed form. */
void oracle_lattice_temperature(int64_t n, const int64_t *rowptr, const int32_t *col,
                                const double *v, const double *mass_of_atom, int dof_mode,
                                double *Tl, double *Kself) {
  const double mvv = o_mvv_ev();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t len = rowptr[i + 1] - rowptr[i] + 1;
    double msum = 0.0, px = 0.0, py = 0.0, pz = 0.0;
    for (int64_t t = -1; t < len - 1; ++t) {
      int64_t j = (t < 0) ? i : col[rowptr[i] + t];
      double m = mass_of_atom[j];
      msum += m;
      px += m * v[3 * j + 0];
      py += m * v[3 * j + 1];
      pz += m * v[3 * j + 2];
    }
    double vcx = px / msum, vcy = py / msum, vcz = pz / msum;
    double ke = 0.0;
    for (int64_t t = -1; t < len - 1; ++t) {
      int64_t j = (t < 0) ? i : col[rowptr[i] + t];
      double dx = v[3 * j + 0] - vcx, dy = v[3 * j + 1] - vcy, dz = v[3 * j + 2] - vcz;
      ke += 0.5 * mass_of_atom[j] * (dx * dx + dy * dy + dz * dz) * mvv;
    }
    double dof_n = (dof_mode == 1) ? (double)(len - 1) : (double)len;
    Tl[i] = (dof_n > 0.0) ? ke / (1.5 * O_KB * dof_n) : 0.0;
    double vi2 = v[3 * i + 0] * v[3 * i + 0] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
    Kself[i] = 0.5 * mass_of_atom[i] * vi2 * mvv;
  }
}

/* ------------------------------------------------------------------------ */
/* Pair term of Eq. HeatTransport, literally: with theta_i = a, theta_j = b,
 * Delta e_ji = -(theta_j - theta_i) and Delta e_ij = -(theta_i - theta_j),
 *   f(a, b) = b (1 - a) exp(a - b) - a (1 - b) exp(b - a).
 * Evaluating f(b, a) performs the same two products in swapped roles, so
 * f(b, a) == -f(a, b) bit for bit.  Pins: antisymmetry, f(a, a) == 0,
 * linearisation slope 1 - 2a(1 - a). */
double oracle_pair_flux(double a, double b) {
  double gain = b * (1.0 - a) * exp(a - b);
  double loss = a * (1.0 - b) * exp(b - a);
  return gain - loss;
}

/* The pair-flux sum of Eq. HeatTransport for every atom, in list order:
 * F_i = sum_j f(theta_i, theta_j), so that d theta_i / dt = K F_i (flux part). */
void oracle_flux_sum(int64_t n, const int64_t *rowptr, const int32_t *col, const double *theta, double *F) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) acc += oracle_pair_flux(theta[i], theta[col[e]]);
    F[i] = acc;
  }
}

/* Partial derivative of the pair term in its first argument, from the same
 * two-exponential form: d/da [b (1 - a) e^{a-b} - a (1 - b) e^{b-a}]
 *   = -b e^{a-b} + b (1 - a) e^{a-b} - (1 - b) e^{b-a} + a (1 - b) e^{b-a}
 *   = -( a b e^{a-b} + (1 - a)(1 - b) e^{b-a} ).
 * Pins: central differences of oracle_pair_flux. */
double oracle_pair_dflux_a(double a, double b) {
  return -(a * b * exp(a - b) + (1.0 - a) * (1.0 - b) * exp(b - a));
}

/* Transposed Jacobian of the flux sum applied to lam (the adjoint of one
 * flux evaluation): out_m = sum_i lam_i dF_i/dtheta_m, with
 * F_i = sum_{j in row i} f(theta_i, theta_j).  Written as the plain double sum
 * over rows i and their entries, not in any symmetrised form, so it holds for
 * any list.  Pins: <u, J v> by central differences of oracle_flux_sum. */
void oracle_flux_vjp(int64_t n, const int64_t *rowptr, const int32_t *col, const double *theta,
                     const double *lam, double *out) {
  for (int64_t m = 0; m < n; ++m) out[m] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = col[e];
      /* dF_i/dtheta_i gains d_a f(theta_i, theta_j); dF_i/dtheta_j gains
       * d_b f(theta_i, theta_j) = -d_a f(theta_j, theta_i) (f is odd) */
      out[i] += lam[i] * oracle_pair_dflux_a(theta[i], theta[j]);
      out[j] -= lam[i] * oracle_pair_dflux_a(theta[j], theta[i]);
    }
}

/* Optional time-dependent source (Sec. 5, Eq. LaserIntesity), a Gaussian pulse
 * absorbed with exponential decay below the irradiated surface:
 *   S(depth, t) = (F / l_p) exp(-depth / l_p) exp(-(t - t0)^2 / (2 s^2)) / (s sqrt(2 pi))
 * [W m^-3], which raises T at rate S / C_e. */
typedef struct {
  int on;
  double fluence_Jm2, lp_A, t0_fs, sigma_fs;
} oracle_source;

/* n_sub explicit forward-Euler substeps of Eq. HeatTransport (Jacobi: every
 * atom reads the same snapshot theta^n), dt in fs:
 *   T_i += dt * ( Tmax * K * F_i - chi_i * (G/C_e) * (T_i - T_l,i) + q_i(t) )
 * with F_i = sum_j f(theta_i, theta_j) over row i in order, theta = T / Tmax
 * (T_min = 0, Sec. 2).  K is the pair rate of Eq. Kij [1/fs]; cG = G/C_e [1/fs].
 * The energy the electrons hand to atom i's lattice (Eq. RateExchange) is
 * accumulated as A_i += dt * chi_i * VG * (T_i - T_l,i), VG = G * V_atom
 * [eV / (K fs)], using T_i before the update.  E_src (if non-null) receives the
 * source energy V_atom * C_e * q_i * dt summed over atoms and substeps.
 * chi_i = 0 switches the coupling off for atom i (Eq. Xi guard).
 * Returns the number of substeps done, or -(substep+1) if some theta left
 * [0, 1] or became NaN. */
/* Distance weights of the pair rates (an optional variant; the paper uses one
 * rate K for every pair of the list): w_ij = S2 / (n_shell r_ij^2), the weight
 * b^2 / r^2 renormalised so that an ideal shell of n_shell neighbours with
 * second moment S2 = sum_j r_j^2 keeps sum_j w_j r_j^2 = S2.  r_ij^2 is the exact
 * squared minimum-image distance on the quantised grid (units 2^-40 A^2), one
 * weight per entry of the list.  Pins: the two FCC shells at r_c = 4 A get
 * 4/3 and 2/3; symmetry; a sin mode decays at the weighted lattice sum. */
void oracle_pair_weights(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *q,
                         const int64_t *Lq, const int32_t *periodic, double S2_A2, int32_t n_shell,
                         double *w) {
  const double S2q = S2_A2 * 1099511627776.0; /* A^2 -> grid units 2^-40 A^2 */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int64_t j = col[e];
      int64_t d2 = 0;
      for (int k = 0; k < 3; ++k) {
        const int64_t d = o_disp((int64_t)q[3 * j + k] - (int64_t)q[3 * i + k], Lq[k], periodic[k]);
        d2 += d * d;
      }
      w[e] = S2q / ((double)n_shell * (double)d2);
    }
}

/* ------------------------------------------------------------------------ */
/* Interatomic forces for the lattice side of Eq. Motion (F_i; the paper uses an
 * EAM potential, not available here): a Morse pair potential
 *   phi(r) = D [exp(-2 alpha (r - r0)) - 2 exp(-alpha (r - r0))]
 * in shifted-force form on the neighbour list (r <= r_c):
 *   phi_sf(r) = phi(r) - phi(r_c) - (r - r_c) phi'(r_c),
 * so that energy and force both vanish at the cutoff.  Displacements are the
 * exact integer minimum-image differences of the quantised positions.
 *   F_i = sum_j phi_sf'(r_ij) (x_j - x_i) / r_ij   [eV/A],
 *   E_i = (1/2) sum_j phi_sf(r_ij)                 [eV].
 * Pins: F = -grad E by central differences; sum_i F_i = 0; a perfect FCC lattice
 * has F = 0 and E_i = (12 phi_sf(a/sqrt2) + 6 phi_sf(a)) / 2; energy of a
 * velocity-Verlet run conserved to O(dt^2). */
void oracle_morse(double r, double D, double alpha, double r0, double *phi, double *dphi) {
  const double e1 = exp(-alpha * (r - r0));
  *phi = D * (e1 * e1 - 2.0 * e1);
  *dphi = -2.0 * alpha * D * (e1 * e1 - e1);
}

void oracle_forces(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *q,
                   const int64_t *Lq, const int32_t *periodic, double D, double alpha, double r0,
                   double rc, double *F, double *E) {
  double pc, dpc;
  oracle_morse(rc, D, alpha, r0, &pc, &dpc);
  const double g = 1.0 / 1048576.0;   /* grid unit [A] */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double f[3] = {0.0, 0.0, 0.0}, e = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int64_t j = col[p];
      double d[3];
      for (int k = 0; k < 3; ++k)
        d[k] = g * (double)o_disp((int64_t)q[3 * j + k] - (int64_t)q[3 * i + k], Lq[k], periodic[k]);
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double ph, dph;
      oracle_morse(r, D, alpha, r0, &ph, &dph);
      const double phs = ph - pc - (r - rc) * dpc;
      const double dphs = dph - dpc;
      for (int k = 0; k < 3; ++k) f[k] += dphs * d[k] / r;
      e += 0.5 * phs;
    }
    for (int k = 0; k < 3; ++k) F[3 * i + k] = f[k];
    E[i] = e;
  }
}

/* Velocity-Verlet half kick: v_i += (dt / (m_i)) F_i, with F in eV/A, m in amu,
 * v in A/fs (1 eV/(A amu) = 1/o_mvv_ev() A/fs^2). */
void oracle_kick(int64_t n, double *v, const double *F, const double *mass_of_atom, double dt) {
  const double mvv = o_mvv_ev();
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) v[3 * i + k] += dt * F[3 * i + k] / (mass_of_atom[i] * mvv);
}

/* Optional fixed-temperature border (a Dirichlet condition on T_e, as the
 * 300 K border shell of the paper's cascade runs, Sec. 5): where Tfix[i] is not
 * NaN, atom i is an electron reservoir held at Tfix[i].  Every substep is first
 * taken for all atoms as above (so a border atom exchanges pair fluxes and
 * coupling energy with its T held at Tfix[i]); then each border atom is put back
 * to Tfix[i] and the change it would have made, T_new - Tfix[i], is added to
 * *Eres_T (kelvin; times V_atom C_e it is the energy the reservoir absorbed). */
int oracle_substeps(int64_t n, const int64_t *rowptr, const int32_t *col, double *T,
                    const double *Tl, const uint8_t *chi, double *A, int n_sub, double dt,
                    double Tmax, double K, double cG, double VG, const double *depth,
                    const double *src, double Ce_SI, double vatom_A3, double t_start,
                    double *E_src, const double *Tfix, double *Eres_T, const double *pw) {
  double *theta = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  double *Tn = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  if (!theta || !Tn) { free(theta); free(Tn); return -1000000; }
  oracle_source S = {0, 0, 0, 0, 0};
  if (src) { S.on = (src[0] != 0.0); S.fluence_Jm2 = src[1]; S.lp_A = src[2]; S.t0_fs = src[3]; S.sigma_fs = src[4]; }
  double esrc = 0.0;
  int status = n_sub;
  for (int s = 0; s < n_sub; ++s) {
    double t = t_start + dt * (double)s;
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
      theta[i] = T[i] / Tmax;
      if (!(theta[i] >= 0.0 && theta[i] <= 1.0)) bad = 1;
    }
    if (bad) { status = -(s + 1); break; }
    double pulse = 0.0;
    if (S.on) {
      double sig_s = S.sigma_fs * 1.0e-15;
      double dtp = (t - S.t0_fs) / S.sigma_fs;
      /* W m^-3 at depth 0 */
      pulse = S.fluence_Jm2 / (S.lp_A * 1.0e-10) * exp(-0.5 * dtp * dtp) /
              (sig_s * sqrt(2.0 * M_PI));
    }
    double esrc_step = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : esrc_step)
    for (int64_t i = 0; i < n; ++i) {
      double F = 0.0;
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
        F += (pw ? pw[p] : 1.0) * oracle_pair_flux(theta[i], theta[col[p]]);
      double dTdt = Tmax * K * F;
      if (chi[i]) {
        dTdt -= cG * (T[i] - Tl[i]);
        A[i] += dt * VG * (T[i] - Tl[i]);
      }
      if (S.on) {
        double Sw = pulse * exp(-depth[i] / S.lp_A);        /* W m^-3 */
        dTdt += Sw / Ce_SI * 1.0e-15;                        /* K / fs */
        esrc_step += Sw * vatom_A3 * 1.0e-30 * dt * 1.0e-15 / O_EV; /* eV */
      }
      Tn[i] = T[i] + dt * dTdt;
    }
    esrc += esrc_step;
    if (Tfix) {
      double absorbed = 0.0;
      for (int64_t i = 0; i < n; ++i)
        if (Tfix[i] == Tfix[i]) {
          absorbed += Tn[i] - Tfix[i];
          Tn[i] = Tfix[i];
        }
      if (Eres_T) *Eres_T += absorbed;
    }
    memcpy(T, Tn, sizeof(double) * (size_t)n);
  }
  if (E_src) *E_src += esrc;
  free(theta); free(Tn);
  return status;
}

/* ------------------------------------------------------------------------ */
/* LOCAL per-atom form of Eq. HeatTransport (Sec. 2: "C_e = lambda T_e",
 * "kappa_e = kappa0 T_e / T_lat", evaluated per atom instead of at the system
 * means).  Every atom carries its own heat capacity C_e,i = min(gamma T_i, cap)
 * and conductivity kappa_i = kappa0 T_i / T_lat (kappa_mode 1; kappa0 in mode 0,
 * T_lat the system's classical lattice temperature of the MD step).  The pair
 * rate of Eq. Kij, K_ij C_e = 2 d kappa / (Z b^2), becomes a pair energy rate
 * with the pair-averaged kappa_ij = (kappa_i + kappa_j) / 2, so that what atom i
 * gains from j is exactly what j loses to i:
 *   q_ij = (2 d / S2) kappa_ij T_max f(theta_i, theta_j) w_ij           [W m^-3]
 *   e_i  = dt [ sum_j q_ij - chi_i G (T_i - T_l,i) + S_i(t) ]           [J m^-3]
 * The explicit step advances the electron energy density of each atom,
 * U(T) = int_0^T C_e dT' (gamma T^2 / 2 below T_c = cap / gamma, linear above),
 * U_i' = U(T_i) + e_i, and returns T_i' = U^{-1}(U_i') in closed form.  To first
 * order this is C_e,i dT_i = e_i; advancing U keeps sum_i U_i exact (the energy
 * form).  Jacobi: every atom reads the previous substep.  A_i, the energy handed
 * to the lattice, and the laser source are those of oracle_substeps.  Border
 * atoms (Tfix finite) keep Tfix and the energy they would have gained,
 * V_atom dt e_i, goes to *Eres_eV.
 * Pins: conservation of sum_i U_i; relaxation of an isolated periodic lattice
 * to U^{-1}(mean U); small-mode decay at the lattice sum with K = 2 d kappa0 /
 * (gamma S2 T_lat); the coupling-only closed form of gamma T dT/dt = -G (T -
 * T_l); above the cap with constant kappa, equal to oracle_substeps. */
static double o_ue(double T, double gamma, double cap) {
  if (cap > 0.0 && gamma * T > cap) {
    const double Tc = cap / gamma;
    return 0.5 * cap * Tc + cap * (T - Tc);
  }
  return 0.5 * gamma * T * T;
}

static double o_ue_inv(double U, double gamma, double cap) {
  if (cap > 0.0) {
    const double Tc = cap / gamma;
    const double Uc = 0.5 * cap * Tc;
    if (U > Uc) return Tc + (U - Uc) / cap;
  }
  return sqrt(2.0 * U / gamma);   /* NaN for U < 0: caught by the range test */
}

double oracle_ce_energy(double T, double gamma, double cap) { return o_ue(T, gamma, cap); }
double oracle_ce_energy_inv(double U, double gamma, double cap) { return o_ue_inv(U, gamma, cap); }

int oracle_substeps_local(int64_t n, const int64_t *rowptr, const int32_t *col, double *T,
                          const double *Tl, const uint8_t *chi, double *A, int n_sub, double dt,
                          double Tmax, double kappa0, int kappa_mode, double Tlat, int dim_d,
                          double S2_A2, double gamma, double cap, double G, double vatom_A3,
                          const double *depth, const double *src, double t_start, double *E_src,
                          const double *Tfix, double *Eres_eV, const double *pw) {
  double *theta = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  double *Tn = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  if (!theta || !Tn) { free(theta); free(Tn); return -1000000; }
  oracle_source S = {0, 0, 0, 0, 0};
  if (src) { S.on = (src[0] != 0.0); S.fluence_Jm2 = src[1]; S.lp_A = src[2]; S.t0_fs = src[3]; S.sigma_fs = src[4]; }
  const double dts = dt * 1.0e-15;                   /* s */
  const double geo = 2.0 * (double)dim_d / (S2_A2 * 1.0e-20);   /* 2 d / (Z b^2)  [m^-2] */
  const double V = vatom_A3 * 1.0e-30;               /* m^3 */
  double esrc = 0.0, eres = 0.0;
  int status = n_sub;
  for (int s = 0; s < n_sub; ++s) {
    double t = t_start + dt * (double)s;
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
      theta[i] = T[i] / Tmax;
      if (!(theta[i] >= 0.0 && theta[i] <= 1.0)) bad = 1;
    }
    if (bad) { status = -(s + 1); break; }
    double pulse = 0.0;
    if (S.on) {
      double sig_s = S.sigma_fs * 1.0e-15;
      double dtp = (t - S.t0_fs) / S.sigma_fs;
      pulse = S.fluence_Jm2 / (S.lp_A * 1.0e-10) * exp(-0.5 * dtp * dtp) / (sig_s * sqrt(2.0 * M_PI));
    }
    double esrc_step = 0.0, eres_step = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : esrc_step, eres_step)
    for (int64_t i = 0; i < n; ++i) {
      const double ki = kappa_mode == 1 ? kappa0 * T[i] / Tlat : kappa0;
      double P = 0.0;                                  /* W m^-3 */
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        const int32_t j = col[p];
        const double kj = kappa_mode == 1 ? kappa0 * T[j] / Tlat : kappa0;
        const double kij = 0.5 * (ki + kj);
        P += (pw ? pw[p] : 1.0) * geo * kij * Tmax * oracle_pair_flux(theta[i], theta[j]);
      }
      if (chi[i]) {
        P -= G * (T[i] - Tl[i]);
        A[i] += dts * G * V * (T[i] - Tl[i]) / O_EV;
      }
      if (S.on) {
        double Sw = pulse * exp(-depth[i] / S.lp_A);
        P += Sw;
        esrc_step += Sw * V * dts / O_EV;
      }
      if (Tfix && Tfix[i] == Tfix[i]) {
        eres_step += P * dts * V / O_EV;
        Tn[i] = Tfix[i];
      } else {
        Tn[i] = o_ue_inv(o_ue(T[i], gamma, cap) + P * dts, gamma, cap);
      }
    }
    esrc += esrc_step;
    eres += eres_step;
    memcpy(T, Tn, sizeof(double) * (size_t)n);
  }
  if (E_src) *E_src += esrc;
  if (Eres_eV) *Eres_eV += eres;
  free(theta); free(Tn);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11): ten rounds of two 32x32->64 multiplications with the round keys
 * bumped by the Weyl constants.  Pins: published known-answer vectors. */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three standard normals for atom `id` at MD step `step`: counter
 * (id lo, id hi, step lo, step hi), key (seed lo, seed hi); uniforms from the
 * top 24 bits of each word, u = (x + 1/2) / 2^24 in (0, 1); Box-Muller in
 * double precision. */
void oracle_gauss3(uint64_t id, uint64_t step, uint64_t seed, double g[3]) {
  uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step, (uint32_t)(step >> 32)};
  uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  oracle_philox4x32_10(c, k, r);
  double u[4];
  for (int m = 0; m < 4; ++m) u[m] = ((double)(r[m] >> 8) + 0.5) / 16777216.0;
  double r1 = sqrt(-2.0 * log(u[0]));
  double r2 = sqrt(-2.0 * log(u[2]));
  g[0] = r1 * cos(2.0 * M_PI * u[1]);
  g[1] = r1 * sin(2.0 * M_PI * u[1]);
  g[2] = r2 * cos(2.0 * M_PI * u[3]);
}

/* Electron -> lattice hand-over once per MD step (Eqs. Motion, WorkDone, Xi).
 * Arrays in original atom order.  For each atom with chi_i = 1 the lattice
 * receives exactly the energy A_i the electrons gave up:
 *   mode 0 (damping, the paper's choice): v_i <- s v_i, s^2 = (K_i + A_i) / K_i.
 *     Integrating m dv/dt = xi m v with xi of Eq. Xi over the step gives this
 *     scaling; it transfers A_i exactly.
 *   mode 1 (Langevin): trial v* = v e^{-g dt} + sqrt(kB T_e,i (1 - e^{-2 g dt}) / m) eta,
 *     g = G V_atom / (3 kB), eta from oracle_gauss3; then v_i <- v* sqrt((K_i + A_i) / K*),
 *     so the random force and friction act and the exchanged energy is A_i.
 * If K_i + A_i < 0 the atom is stopped (lattice hands over only K_i) and the
 * difference is returned to the electrons: T_i += (A_i - dKE_i) / VC,
 * VC = V_atom C_e [eV/K].  frozen != 0 leaves v untouched (the lattice is a
 * bookkeeping sink) and reports dKE_i = A_i.  A is reset to zero.
 * dKE (out) holds each atom's kinetic-energy change.  Returns the number of
 * atoms that had to be stopped. */
/* Electronic stopping (the cascade runs of Sec. 5: a friction force on atoms
 * with kinetic energy above a cut, 10 eV there, with SRIM's stopping power): here
 * m dv/dt = -beta m v above E_cut (a stopping power proportional to the speed),
 * integrated over the MD step: the atom's kinetic energy K loses
 * K (1 - exp(-2 beta dt_md)), and its own electrons gain that energy, through the
 * same exact hand-over as A_i (the target kinetic energy is K + A_i minus the
 * stopping loss; whatever the lattice does not take goes back to T_i).
 * rng_id (may be NULL): the id that keys atom i's Gaussian numbers in mode 1
 * (NULL: i itself); a slab domain of a decomposed system passes its atoms'
 * global ids, so that they draw what the undivided system draws. */
int64_t oracle_couple(int64_t n, double *v, const double *mass_of_atom, double *A, double *T,
                      const uint8_t *chi, int mode, int frozen, uint64_t seed, uint64_t md_step,
                      double dt_md, double gamma_fs, double VC, double *dKE, double stop_beta,
                      double stop_ecut, const int64_t *rng_id) {
  const double mvv = o_mvv_ev();
  int64_t stopped = 0;
#pragma omp parallel for schedule(static) reduction(+ : stopped)
  for (int64_t i = 0; i < n; ++i) {
    dKE[i] = 0.0;
    if (!chi[i]) { A[i] = 0.0; continue; }
    if (frozen) { dKE[i] = A[i]; A[i] = 0.0; continue; }
    double m = mass_of_atom[i];
    double *vi = v + 3 * i;
    double K0 = 0.5 * m * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]) * mvv;
    double target = K0 + A[i];
    const int slowed = stop_beta > 0.0 && K0 > stop_ecut;
    if (slowed) target -= K0 * (1.0 - exp(-2.0 * stop_beta * dt_md));
    if (target < 0.0) { target = 0.0; stopped += 1; }
    double w[3] = {vi[0], vi[1], vi[2]};
    if (mode == 1) {
      double g[3];
      oracle_gauss3(rng_id ? (uint64_t)rng_id[i] : (uint64_t)i, md_step, seed, g);
      double e1 = exp(-gamma_fs * dt_md);
      double e2 = exp(-2.0 * gamma_fs * dt_md);
      double sig = sqrt(O_KB * T[i] * (1.0 - e2) / (m * mvv));
      for (int k = 0; k < 3; ++k) w[k] = vi[k] * e1 + sig * g[k];
    }
    double Kw = 0.5 * m * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]) * mvv;
    double s = (Kw > 0.0) ? sqrt(target / Kw) : 0.0;
    for (int k = 0; k < 3; ++k) vi[k] = w[k] * s;
    dKE[i] = target - K0;   /* the kinetic energy after scaling is the target */
    if (target == 0.0 || slowed) T[i] += (A[i] - dKE[i]) / VC;
    A[i] = 0.0;
  }
  return stopped;
}
