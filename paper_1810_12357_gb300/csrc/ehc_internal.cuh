// ehc_internal.cuh -- device data layout and kernel launchers of libehc.
//
// Layout in HBM (N atoms, W = neighbour-table width):
//   atoms are kept in a cell-sorted order s (cells x-fastest, within a cell by
//   original id); perm[s] = original id, inv_perm[original] = s.
//   nbr   int32 [W][N]  slot-major: nbr[k*N + s] = k-th neighbour of s (sorted index),
//                       a row lists its neighbours by ascending original id
//   pidx  u32 [W/2][ps] the same neighbours as 16-bit indices into the row tile,
//                       two per word; ps = N rounded up to a multiple of 4
//   cnt   uint8 [N]     neighbour count of s
//   T     double[N]     electronic temperature (FP64 state), sorted order
//   dmir  float [2][N]  (T - Tref)/Tmax mirror, double-buffered across substeps
//   A     double[N]     energy handed from electrons to the lattice this MD step [eV]
//   Tl_f  float [N]     local lattice temperature (negative: atom below the guard)
//   Tl_d  double[N]     same in FP64 (for the FP64 flux path and diagnostics)
//   v_s   VelQ  [N]     velocity on a 2^-48 A/fs integer grid and |v|^2 (FP64), sorted
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ehc.h"

namespace ehc {

constexpr int kMaxTypes = 16;
constexpr int kMaxWidth = 64;

enum DevErr : int32_t {
  ERR_RANGE = 1,         // theta outside [0,1] or NaN
  ERR_NBR_OVERFLOW = 2,  // more neighbours than the table width
  ERR_BOUNDS = 4,        // atom outside a non-periodic extent
  ERR_TIMEOUT = 8,       // bounded wait gave up
  ERR_NEG_KE = 16,       // (informational) kinetic energy could not pay A_i
  ERR_SPEED = 32,        // a velocity component outside the fixed-point range (|v| >= 256 A/fs or NaN)
  ERR_INDEX = 64,        // (EHC_CHECKED builds) a gathered index outside its table
};

// Builds with -DEHC_CHECKED bounds-check every gathered neighbour and tile index:
// an index outside [0, bound) sets ERR_INDEX in the device error word and is
// replaced by 0, so the access stays in bounds (no trap).  Otherwise a no-op.
__device__ __forceinline__ uint32_t checked_index(uint32_t i, uint32_t bound, int32_t *err) {
#ifdef EHC_CHECKED
  if (i >= bound) {
    atomicOr(err, ERR_INDEX);
    return 0u;
  }
#else
  (void)bound;
  (void)err;
#endif
  return i;
}

// ---- exact FP64 conversions on the integer pipes ----
// The FP64 pipe of this GPU retires about two lanes per SM clock, so the
// once-per-MD-step kernels keep it for the arithmetic the ledger needs and do
// scalings by powers of two, roundings to integers, fixed-point sums and range
// tests on the bit patterns.

// round-half-even(x * 2^s) as int64, bit for bit what cvt.rni.s64.f64 gives for
// x * 2^s (an exact scaling): NaN -> 0, out of range -> saturated.
__device__ __forceinline__ long long rint_scaled(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  const unsigned long long frac = b & 0xfffffffffffffull;
  const bool neg = (b >> 63) != 0;
  if (e == 0x7ff && frac != 0) return 0;                        // NaN
  if (e == 0) return 0;                                          // zero, subnormal (|x 2^s| < 1/2 for s < 1000)
  const unsigned long long m = frac | (1ull << 52);
  const int sh = e - 1075 + s;                                   // x 2^s = m 2^sh
  if (sh > 10) return neg ? (long long)0x8000000000000000ull : 0x7fffffffffffffffll;   // |x 2^s| >= 2^63
  unsigned long long r;
  if (sh >= 0) {
    r = m << sh;
  } else if (sh < -54) {
    r = 0;                                                       // |x 2^s| < 1/2
  } else {
    const int k = -sh;                                           // 1..54
    const unsigned long long q = m >> k;
    const unsigned long long rem = m & ((1ull << k) - 1ull);
    const unsigned long long half = 1ull << (k - 1);
    r = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  }
  return neg ? -(long long)r : (long long)r;
}

// |x| < 2^k (false for NaN and infinities)
__device__ __forceinline__ bool abs_below_pow2(double x, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (int)((b >> 52) & 0x7ffu) < 1023 + k;
}

// (hi, lo) += floor(x * 2^96), a double 0 <= x < 2^31 on the 2^-96 fixed-point
// grid (exact: the bits below 2^-96 are dropped), as a 128-bit integer in two
// words; the usual exponents (2^-43 <= x < 2^11) take the branch-free path
__device__ __forceinline__ void fix96_add(unsigned long long &hi, unsigned long long &lo, double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
  const int sh = e - 1075 + 96;                                  // x 2^96 = m 2^sh
  const bool pos = !(b >> 63);
  unsigned long long l = 0, h = 0;
  if (pos && sh >= 0 && sh < 64) {
    l = m << sh;
    h = (m >> 1) >> (63 - sh);                                   // m >> (64 - sh), 0 for sh = 0
  } else if (pos && e != 0) {
    if (sh >= 64) h = m << (sh - 64 < 10 ? sh - 64 : 10);        // outside the stated range: clamped
    else if (sh > -53) l = m >> (-sh);
  }
  const unsigned long long nl = lo + l;
  hi += h + (nl < l ? 1ull : 0ull);
  lo = nl;
}

// the double nearest to a signed 128-bit integer (ties to even)
__device__ __forceinline__ double i128_to_double(__int128 v) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long hi0 = (unsigned long long)(u >> 64);
  const int lz = hi0 ? __clzll((long long)hi0) : 64 + __clzll((long long)(unsigned long long)u);
  u <<= lz;                                                      // top bit at 127
  const unsigned long long top = (unsigned long long)(u >> 64);
  const unsigned long long low = (unsigned long long)u;
  unsigned long long m = top >> 11;                              // 53 bits
  const unsigned long long rb = (top >> 10) & 1ull;              // first dropped bit
  const bool sticky = ((top & 0x3ffull) | low) != 0;
  if (rb && (sticky || (m & 1ull))) ++m;
  int ex = 127 - lz;                                             // value = 1.f * 2^ex
  if (m >> 53) {
    m >>= 1;
    ++ex;
  }
  const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)(ex + 1023) << 52) |
                                  (m & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

// exact float -> double by bit assembly on the integer pipes (zero and
// subnormal inputs give a signed zero); keeps the FP64 pipe for the ledger
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sg = u & 0x80000000u;
  const uint32_t ex = (u >> 23) & 0xffu;
  const uint32_t man = u & 0x7fffffu;
  uint32_t hi = sg, lo = 0u;
  if (ex != 0u) {
    hi = sg | ((ex + 896u) << 20) | (man >> 3);
    lo = man << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// the float nearest to x (ties to even), bit for bit the conversion's result, on
// the integer pipes for |x| in the normal single-precision range (2^-126 up to
// the largest float) and below 2^-150 (a signed zero); subnormal results,
// infinities and NaN take the conversion instruction
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu) - 1023;
  if (e < -150) return __uint_as_float((uint32_t)(b >> 32) & 0x80000000u);
  if (e < -126 || e > 127) return (float)x;
  const uint32_t hi = (uint32_t)((b >> 29) & 0x7fffffu);       // the 23 kept fraction bits
  const uint32_t rem = (uint32_t)b & 0x1fffffffu;              // the 29 dropped ones
  uint32_t r = ((uint32_t)(e + 127) << 23) | hi;
  r += (rem > 0x10000000u || (rem == 0x10000000u && (hi & 1u))) ? 1u : 0u;   // may carry into the exponent
  return __uint_as_float(((uint32_t)(b >> 32) & 0x80000000u) | r);
}

// x as an unevaluated float pair h + l on the integer pipes: h = x truncated to
// 24 significant bits (bit assembly), l = the remaining 29 bits rounded to a
// float (one integer-to-float conversion times a power of two), so that
// |x - (h + l)| <= 2^-48 |x| for 2^-74 <= |x| < 2^127 (below, l = 0: an error
// under 2^-98; below 2^-100, h = 0 too)
__device__ __forceinline__ void split_pair(double x, float &h, float &l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t hw = (uint32_t)(b >> 32);
  const uint32_t sg = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu) - 1023;
  h = __uint_as_float(sg);
  l = h;
  if (e < -100) return;
  h = __uint_as_float(sg | ((uint32_t)(e + 127) << 23) | ((hw & 0xfffffu) << 3) | ((uint32_t)(b >> 29) & 7u));
  const uint32_t t = (uint32_t)b & 0x1fffffffu;     // x - h = t 2^(e - 52)
  if (e >= -74) l = __fmul_rn(__uint2float_rn(t), __uint_as_float(sg | ((uint32_t)(e - 52 + 127) << 23)));
}

// Sorted velocity of one atom: components on a fixed-point grid of 2^-48 A/fs
// (|v| < 256 A/fs, so sums over an atom and up to 64 neighbours stay exact in
// int64) and |v|^2 in FP64.
constexpr double kVelScale = 281474976710656.0;   // 2^48
constexpr double kVelUnit = 1.0 / kVelScale;
constexpr double kVelMax = 256.0;
struct __align__(32) VelQ {
  long long x, y, z;
  double w;
};

// exact reciprocals of 1..kMaxWidth+1 and of (3/2) k_B times the same counts,
// for the lattice temperature (one rounding instead of a division per atom);
// coefT[k]: the one-type factor from the 2^-96 fixed-point sums of an atom with
// k neighbours to its temperature
struct RecipTab {
  double inv_n[kMaxWidth + 2];
  double inv_dof[kMaxWidth + 2];
  double coefT[kMaxWidth + 2];
};

struct MassTable {
  double m[kMaxTypes];
  int32_t n_types;
};

struct Grid {
  int64_t Lq[3];   // box on the 2^-20 A grid
  int32_t nc[3];   // cells per axis
  int32_t per[3];  // periodic flags
  int64_t rcq;     // cutoff on the grid
  int64_t ncell;
};

// Per-MD-step coefficients read by the substep kernels through a pointer, so
// that captured graphs stay valid when the values change.
struct StepCoef {
  double dtTK;     // dt * Tmax * K
  double dtcG;     // dt * G / C_e
  double dtVG;     // dt * G * V_atom [eV/K]
  double dt;       // substep [fs]
  double invTmax;  // 1 / Tmax
  double Tref;     // mirror reference
  float th_ref;    // Tref / Tmax
  float omt;       // 1 - Tref / Tmax
  float dtK_f;     // dt * K: flux increment of delta = (T - Tref) / Tmax
  float dtcGn_f;   // dt * G / (C_e Tmax)
  float Tmax_f;
  float pad[3];
  // LOCAL per-atom C_e / kappa_e form (ce_mode 1).  State: the electron energy
  // density in units of gamma Tmax^2, u(theta) = theta^2 / 2 below theta_c =
  // T_c / Tmax and theta_c theta - theta_c^2 / 2 above (no cap: theta_c = 0).
  double dtKu;     // dt * 2 d kappa0 / (Z b^2 gamma T_lat) (kappa_mode 1) or / (... gamma Tmax) (mode 0) [1]
  double dtgu;     // dt * G / (gamma Tmax^2) [1/K]
  double thc;      // theta_c (0: no cap)
  double u_ref;    // u(Tref / Tmax): the single-precision state is w = u - u_ref
  float dtKu_f, dtgu_f, thc_f, inv_thc_f;
  float wc_f;      // w at the cap, u(theta_c) - u_ref
  float thsq_f;    // (Tref / Tmax)^2
  int32_t kmode;   // 1: kappa_ij / kappa_scale = (theta_i + theta_j) / 2; 0: 1
  float pad2;
  double dtVGu;    // (double)dtgu_f * V_atom gamma Tmax^2 [eV/K]: the lattice's share, single-precision path
};

// u(theta) and its inverse of the LOCAL form (FP64): energy density per gamma Tmax^2
__device__ __forceinline__ double ue_of(double th, double thc) {
  if (thc > 0.0 && th > thc) return thc * th - 0.5 * thc * thc;
  return 0.5 * th * th;
}
__device__ __forceinline__ double ue_inv(double u, double thc) {
  if (thc > 0.0 && u > 0.5 * thc * thc) return (u + 0.5 * thc * thc) / thc;
  return sqrt(2.0 * u);   // NaN for u < 0: caught by the range checks
}

// Row tiles: a row is the run of cells with the same (cy, cz); its atoms are a
// contiguous range of the sorted order.  Every neighbour of an atom lies in the
// (at most 9, deduplicated) rows around its own, listed in a fixed order.
constexpr int kRowNbr = 9;
constexpr int kTileThreads = 256;   // threads that own atoms (plus one descriptor warp)
constexpr int kTileMinBlocks = 4;
constexpr int kTileMaxBytes = 200 * 1024;   // the tile buffers must fit in this much shared memory


// Arguments of one system for the row-tile substep kernel (device table; one
// entry for a single system, one per replica for a batch).  Pointers stay
// fixed for the life of a context; P is refreshed after every neighbour build.
struct RepArgs {
  int32_t n, ncx, P, nrows;
  int32_t ps, rsv;               // plane stride of pidx (words, a multiple of 4)
  const int32_t *start, *row_nbr;
  const uint32_t *pidx;
  float *dmir[2];
  float *lo;
  double *A;
  const float *uTl, *srcw, *pulse_f;
  float *rrange[2];
  const StepCoef *cf;
  int32_t *err;
  const uint8_t *fix;   // border mask (null: no border)
  double *res;          // border reservoirs (single-precision paths: a float pair per atom, delta units)
  float *uhi;           // LOCAL form: high word of the energy state (lo holds its low word)
  uint32_t *ldmax;      // LOCAL form: ring of the largest |Delta| per substep (float bits)
};

// Arguments of a Chebyshev-window stage launch of the row-tile kernel.  The
// window's change z_j = Y_j - Y_0 is carried separately (single precision
// relative to the change):
//   z_j = z_{j-1} + nu (z_{j-2} - z_{j-1}) - kap z_{j-1} + mt F(Y_{j-1}) + gt F_0,
//   Y_j = Y_0 + z_j (the values the next stage's tiles are copied from),
// values as delta = (T - Tref)/Tmax; optionally F itself into Fout.  The kap and
// F_0 terms belong to the second-order recurrence (F0 null otherwise).
struct StageArgs {
  const float *yin;     // Y_{j-1}: the values the tiles are copied from (padded to ps)
  const float *y0;      // Y_0
  const float *zin;     // z_{j-1} (null: zero, the first stage)
  const float *zprev;   // z_{j-2} (null: zero)
  const float *F0;      // F(Y_0) (null: no gt term)
  float *yout;          // Y_j (null with zout: a flux pass, Fout only)
  float *zout;          // z_j
  float *Fout;          // the pair-flux sum F(Y_{j-1}) per atom, or null
  float *rr[2];         // row value ranges of the stage values (read [parity], write [parity ^ 1])
  float nu, mt, kap, gt;   // nu_j, mut_j tau K, 1 - mu_j - nu_j, gam_j tau K
  // the window's last stage (T1 non-null) also ends the window in FP64:
  // T1 = T0 + Tmax z - dT with the coupling of the window dT = fin (T0 - T_l)
  // (single precision, also into dTc), and Y_j lowered by dT / Tmax
  const double *T0;
  double *T1, *dTc;
  float fin, Tref_f, invTmax_f;
  double Tmax;
};

// Deterministic block-partial reductions.
constexpr int kRedBlocks = 304;   // 2 x 152 SMs
constexpr int kRedThreads = 256;

struct Ctx;

// kernels_build.cu
cudaError_t launch_bin(Ctx &c, const double *x);
cudaError_t launch_sort_cells(Ctx &c);
// v == nullptr: positions, temperatures and types only; launch_gather_vel then
// gathers the velocities (before the lattice temperature)
cudaError_t launch_gather(Ctx &c, const double *v, bool first);
cudaError_t launch_gather_vel(Ctx &c, const double *v);
cudaError_t launch_neighbors(Ctx &c);
cudaError_t launch_lattice_temperature(Ctx &c);
cudaError_t launch_globals(Ctx &c);
cudaError_t launch_unpermute(Ctx &c, const double *src_sorted, double *dst_orig, int mode);
cudaError_t launch_seed(Ctx &c, double cap_SI);
cudaError_t launch_ledger(Ctx &c);
// kernels_substep.cu
cudaError_t launch_substep(Ctx &c, int k, int parity, cudaStream_t s);
cudaError_t launch_split(Ctx &c, cudaStream_t s);
cudaError_t launch_merge(Ctx &c, int parity, cudaStream_t s);
bool tile_path(const Ctx &c);
// the bounded-wait probe (kernels_substep.cu): ERR_TIMEOUT into *flag if the wait runs out
cudaError_t launch_wait_probe(uint32_t polls, int complete, int32_t *flag, cudaStream_t st);
// ghost exchange (kernels_halo.cu): T of caller-order atoms idx[0..m) into out; overwrite them
cudaError_t launch_get_at(Ctx &c, const int32_t *idx, int64_t m, double *out);
cudaError_t launch_set_at(Ctx &c, const int32_t *idx, int64_t m, const double *vals);
// sum T and sum of the kinetic energy [eV] over the listed atoms into out[0..1]
// (part: 2 x 152 doubles of block sums)
cudaError_t launch_sums_at(Ctx &c, const int32_t *idx, int64_t m, double *part, double *out);
// the LOCAL form's substeps run on the row tiles (single precision, no laser source)
bool local_tile(const Ctx &c);
// tile capacity tb with headroom for the largest staged tile, the shared-memory
// opt-in and the resident grid of each index width (9 and 16 words); false:
// the buffers do not fit
bool tile_size(int32_t staged, int num_sms, int32_t *tb, int32_t grid[2], int32_t grid128[2]);
cudaError_t launch_tile_worklist(const RepArgs *reps, const int2 *work, int32_t nwork, int32_t tb, int grid,
                                 int pairs, int parity, int k, int nt, cudaStream_t st);
cudaError_t launch_cheb_stage(Ctx &c, const StageArgs &sa, int parity, cudaStream_t st);
// kernels_window.cu (Chebyshev window propagator)
cudaError_t cheb_mirror(Ctx &c, const double *T, float *y);
cudaError_t cheb_accept(Ctx &c, const double *dTc);
cudaError_t cheb_residual(Ctx &c, const double *T0, const double *T1, const float *F0, const float *F1, double tau,
                          float *part, float *out);
int cheb_blocks(int64_t n);
// kernels_wtrain.cu (training of the window's stage coefficients)
constexpr int kMaxStages = 32;
// per-stage buffers of a window kept for the backward sweep: z[j] = Y_j - Y_0,
// F[j] = F(Y_{j-1}) (F[1] = F(Y_0)), lam[j] = dL/dz_j, j = 1..s
struct WtTab {
  const float *z[kMaxStages + 1];
  const float *F[kMaxStages + 1];
  const float *lam[kMaxStages + 1];
};
// stage coefficients as the kernels take them: a_j = mut_j tau K, g_j = gam_j tau K
struct WtCoef {
  float nu[kMaxStages + 1], kap[kMaxStages + 1], a[kMaxStages + 1], g[kMaxStages + 1];
};
cudaError_t wt_stages(Ctx &c, int s, const WtCoef &k, const float *y0, const WtTab &t);
cudaError_t wt_backward(Ctx &c, int s, const WtCoef &k, const float *y0, const WtTab &t, const double *T0,
                        const double *T1, int loss_power, double *lpart, double *dpart, double tauK,
                        const float *c0, float *gc, float *gd, float *loss);
// rollout of nwin chained windows: y0[0..nwin] the window starts (y0[w + 1] = y0[w]
// + z_s of window w), t[w] their stage buffers, Tt[w] the targets (sorted, FP64),
// lam[1..s] shared adjoint buffers; Lam, mu, gs, tmp: n floats of work space; zero:
// n zero floats; lpart: nwin x wt_loss_partials
cudaError_t wt_rollout(Ctx &c, int s, const WtCoef &k, int nwin, const float *const *y0, const WtTab *t,
                       const double *const *Tt, float *const *lam, float *Lam, float *mu, float *gs, float *tmp,
                       const float *zero, int loss_power, double *lpart, double *dpart, double tauK,
                       const float *c0, float *gc, float *gd, float *loss);
cudaError_t wt_next_start(Ctx &c, const float *y0, const float *zs, float *y1);
size_t wt_dot_partials(int64_t n, int s);
size_t wt_loss_partials(int64_t n);
cudaError_t wt_adam(cudaStream_t st, int np, float *p, float *m, float *v, const float *g, float lr, int t);
cudaError_t wt_end(Ctx &c, const double *T0, const float *zs, double *T1);
// |lambda_max| of the pair-flux Jacobian at the values y by `iters` products with
// J^T (v, u: n floats; part: wt_dot_partials; ss: one double, |J^T v|^2 at the end)
cudaError_t wt_power(Ctx &c, const float *y, const float *zero, float *v, float *u, double *part, double *ss,
                     int iters);
// kernels_nn.cu (learned window propagator)
int nn_blocks(int64_t n);
cudaError_t nn_gather(Ctx &c, const double *Tin, const double *Ttar, double *Ts, double *Ttar_s, float *dm,
                      bool sorted);
cudaError_t nn_forward(Ctx &c, int H, const __nv_bfloat16 *pb, double sigma, int n_w, const float *dm,
                       __nv_bfloat16 *h, const double *Tin, double *Tout, float *dm_out);
cudaError_t nn_grad(Ctx &c, int H, const __nv_bfloat16 *pb, double sigma, int n_w, const float *dm,
                    __nv_bfloat16 *h, const double *Tin, const double *Ttar, float *gphi, float *p2, float *p1,
                    float *grad, float *loss);
cudaError_t nn_adam(cudaStream_t st, int np, float *p, float *m, float *v, const float *g, float lr, int t,
                    __nv_bfloat16 *pb);
cudaError_t nn_params_to_bf16(cudaStream_t st, int np, const float *p, __nv_bfloat16 *pb);
cudaError_t nn_residual(Ctx &c, const float *d0, const float *d1, const double *T0, const double *T1, double tau,
                        float *part, float *out);
cudaError_t nn_couple_window(Ctx &c, const double *T0, double *T1, float *d1, double *dTc, int n_w);
cudaError_t nn_accept(Ctx &c, const double *dTc);
// kernels_gnn.cu (learned corrector of the window propagator: node width 64,
// tensor-core node MLP, 6336 parameters)
constexpr int kGnnParams = 6336;
constexpr int kCandWidth = 48;   // candidate slots per atom of the skin path
int gnn_mlp_blocks(Ctx &c);
int gnn_edge_blocks(int64_t n);
int gnn_loss_blocks(int64_t n);
size_t gnn_bwd_smem();
cudaError_t gnn_setup(size_t smem);
// corrected window result: y the window result's mirror (sorted), T (sorted FP64)
// corrected in place, y_out its new mirror (must not alias y), dY (optional) the
// correction; in, u: n x 16 BF16 work arrays
cudaError_t gnn_forward(Ctx &c, const __nv_bfloat16 *wb, double sigma, double kappa, const float *y,
                        __nv_bfloat16 *in, __nv_bfloat16 *u, double *T, float *y_out, double *dY);
// gradient of the window loss mean(((Y^ - T*)/T*)^2) after gnn_forward: Yh the
// corrected result, Ts the target (sorted FP64); the loss into *loss (device)
cudaError_t gnn_backward(Ctx &c, const __nv_bfloat16 *wb, double sigma, double kappa, const float *y,
                         const __nv_bfloat16 *in, const __nv_bfloat16 *u, const double *Yh, const double *Ts,
                         float *G, float *du, double *lpart, double *loss, float *mpart, float *epart, float *grad);
cudaError_t gnn_adam(cudaStream_t st, float *p, float *m, float *v, const float *g, float lr, int t,
                     __nv_bfloat16 *pb);
cudaError_t gnn_params_to_bf16(cudaStream_t st, const float *p, __nv_bfloat16 *pb);
// kernels_border.cu (fixed-temperature border)
int border_red_blocks();
cudaError_t border_flush(Ctx &c, double *out, bool clear);   // sum of the reservoirs into *out (device)
cudaError_t border_apply(Ctx &c);                            // mask of the current sort order, T to T_b
// kernels_couple.cu
cudaError_t launch_couple(Ctx &c, double *v, double dt_md);
cudaError_t launch_drift(Ctx &c, double *x, const double *v, double dt);
// lattice side (kernels_md.cu): shifted-force Morse forces of the last build's
// positions into F (caller order, [N,3]) and their energy into *out; v += dt F / m;
// the largest |v| into *out
int md_force_blocks(int64_t n);
cudaError_t launch_forces(Ctx &c, double *F, double *part, double *out);
cudaError_t launch_kick(Ctx &c, double *v, const double *F, double dt);
cudaError_t launch_vmax(Ctx &c, const double *v, double *part, int nb, double *out);
cudaError_t launch_philox_normals(const int64_t *ids, int64_t n, uint64_t step, uint64_t seed,
                                  double *out, cudaStream_t s);

struct Ctx {
  ehc_params p;
  int64_t n = 0;
  int32_t W = 32;
  double box[3];
  Grid g;
  MassTable mt;
  double vatom = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t pulse_ev = nullptr;
  // host-buffer MD step: the velocity upload and download run on io_stream,
  // ordered against the context stream by io_ev
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_ev[4] = {nullptr, nullptr, nullptr, nullptr};

  // device buffers
  int32_t *type_orig = nullptr;  // caller's type index per atom (original order), or null
  int8_t *type_s = nullptr;
  int4 *q_orig = nullptr;        // quantised position + cell id, original order
  int32_t *cell_count = nullptr; // [ncell + 1]
  int32_t *cell_start = nullptr; // [ncell + 1]
  int32_t *cell_fill = nullptr;  // [ncell]
  int32_t *scan_tmp = nullptr;   // block sums of the scan
  int32_t *perm = nullptr;
  int32_t *perm_raw = nullptr;   // [N] the cells' atoms in scatter order, before the sort by id
  int32_t *inv_perm[2] = {nullptr, nullptr};
  int cur_inv = 0;
  int4 *q_s = nullptr;           // sorted positions + cell id
  VelQ *v_s = nullptr;           // sorted velocities (fixed point) and |v|^2
  int32_t *nbr = nullptr;        // [W][N]
  uint32_t *pidx = nullptr;      // [W/2][ps] pairs of 16-bit tile-local neighbour indices
  int64_t ps = 0;                // plane stride of pidx: N rounded up to a multiple of 4
  int32_t *row_nbr = nullptr;    // [nrows][9] neighbour rows, -1 padded
  int64_t nrows = 0;
  uint8_t *cnt = nullptr;
  double *T[2] = {nullptr, nullptr};   // T[tcur] is the state
  int tcur = 0;
  float *dmir[2] = {nullptr, nullptr};  // hi part of delta = (T - Tref)/Tmax, double-buffered
  float *dlo = nullptr;          // lo part of delta (float-float state of the FP32 path)
  // LOCAL form (ce_mode 1), single-precision path: the state is the float pair
  // (uhi, dlo) of w = u - u_ref; dmir holds delta = theta - Tref/Tmax rebuilt from it
  bool local = false;
  float *uhi = nullptr;
  uint32_t *ldmax = nullptr;   // [3] ring of the largest |Delta| per substep (float bits)
  float *uTl = nullptr;          // Tref - T_l,i (NaN: atom below the guard)
  double *abuf[2] = {nullptr, nullptr};
  double *A = nullptr;           // one of abuf
  double *A_tmp = nullptr;       // the other
  float *Tl_f = nullptr;
  double *Tl_d = nullptr;
  double *depth_orig = nullptr;
  float *srcw = nullptr;         // exp(-depth / l_p), sorted (single-precision path)
  double *srcw_d = nullptr;      // the same in FP64 (double-precision path)
  double *pulse = nullptr;       // per-substep source rate factors [max_sub] (K/fs, FP64 path)
  double *pulse_host = nullptr;  // pinned staging
  float *pulse_f = nullptr;      // dt * rate / Tmax per substep (FP32 path)
  float *pulse_f_host = nullptr;
  int32_t max_sub = 0;
  double *dKE = nullptr;
  double *partials = nullptr;    // [kRedBlocks * 6]
  double *scal = nullptr;        // device scalars [16]
  double *scal_host = nullptr;   // pinned mirror [16]
  int32_t *err = nullptr;        // device error word
  int32_t *maxcnt = nullptr;     // device max count (err + 1)
  int32_t *maxstaged = nullptr;  // largest staged row-tile size (err + 2)
  int32_t *maxrow = nullptr;     // longest row (err + 3); err + 4: the candidate list's rebuild flag
  // neighbour candidates with a skin (ehc_params.skin_A > 0): atoms within r_c + skin
  // at the last candidate build, original ids in visit order [N][kCandWidth] by original id, their
  // counts, and the quantised positions of that build
  int64_t skin_q = 0;            // skin on the 2^-20 A grid (0: full search every build)
  bool cand_valid = false;
  int32_t *cand = nullptr;
  uint8_t *ccnt = nullptr;
  int4 *q_ref = nullptr;
  // ids keying each caller-order atom's Langevin stream (null: the caller index);
  // set by ehc_set_rng_ids, allocated there on first use
  int64_t *rng_id = nullptr;
  int32_t staged_max = 0;
  int32_t row_max = 0;
  int32_t tile_floats = 0;       // floats per tile buffer of the row-tile kernel (0: not set up)
  int32_t tile_grid[2] = {0, 0};  // resident CTAs of the row-tile kernel (9 / 16 index words)
  int32_t tile_grid128[2] = {0, 0};  // the same for its 128-thread form
  int32_t tile_nt = 0;           // threads owning atoms chosen by the tuner (0: not tuned yet, 256)
  int32_t tile_q = 4;            // persistent grid of the row-tile kernel in quarters of the resident CTAs
  int32_t tile_q_fixed = 0;      // ehc_params.tile_grid_quarters (0: tuned with the width, or 4)
  int32_t tile_nt_fixed = 0;     // ehc_params.tile_threads (0: tuned)
  int32_t num_sms = 0;
  RepArgs *reps = nullptr;       // device table of the row-tile kernel (this system only)
  int2 *work = nullptr;          // (system, row) work list of the row-tile kernel
  int32_t nwork = 0;
  float *rrange[2] = {nullptr, nullptr};  // [min of every row | max of every row] of each mirror
  float *wgt = nullptr;          // [W][N] pair weights (ehc_params.rate_shell_n > 0), else null
  double *wgt_d = nullptr;       // [W][N] the same weights in FP64 for the FP64 flux path (flux_prec 1), else null
  StepCoef *coef = nullptr;      // device
  StepCoef *coef_host = nullptr; // pinned
  double *x_dev = nullptr, *v_dev = nullptr, *T_out = nullptr;  // staging of the host-buffer step

  // state
  bool have_te = false;
  bool te_orig_order = false;    // T[tcur] still in caller order (before the first build)
  bool built = false;
  bool have_depth = false;
  bool ff_valid = false;         // float-float substep state holds the current temperatures
  bool t_stale = false;          // T[tcur] is behind the float-float state
  int parity = 0;                // mirror buffer holding the current snapshot
  int64_t md_step = 0;           // counter of the Langevin stream (ehc_set_rng_ids may set it)
  int64_t builds = 0;            // neighbour builds so far
  int64_t t_version = 0;         // bumped by everything that changes or reorders T
  int32_t n_max = 0;             // largest neighbour count this MD step
  int32_t dev_err = 0;

  // per-step scalars
  double Te_mean = 0, Tlat = 0, Ce = 0, K = 0, cG = 0, VG = 0, VC = 0, gammaL = 0;
  double stability = 0, wsum = 0;

  // ledger (host, FP64)
  double E_e0 = 0, E_base = 0, ST_base = 0, VC_prev = -1, E_src = 0;
  double Tmin = 0;       // smallest T_e at the build (LOCAL form's stability number)
  double cap_si = 0;     // cap of C_e per unit volume [J m^-3 K^-1] (0: none)
  double *md_part = nullptr;  // block sums of the force kernel's energy

  // captured substep loops, keyed by everything a launch bakes in
  // fixed-temperature border: tfix_orig (caller order, NaN = free) set by
  // ehc_set_border takes effect at the next build (border_next), which makes
  // the sorted mask bmask; bres holds the reservoirs, 8 bytes per atom: a float
  // pair in delta units on the single-precision paths, a double in kelvin on the
  // FP64 path; bnd_part sum partials
  double *tfix_orig = nullptr;
  bool border_next = false, has_border = false;
  uint8_t *bmask = nullptr;
  double *bres = nullptr, *bnd_part = nullptr;
  double E_res = 0.0;   // energy the border absorbed in closed MD steps [eV]
  struct GraphEntry {
    int n_sub, parity, tcur, abuf, path, pairs, tile, nt, border;
    cudaGraphExec_t exec;
    uint64_t last_use;
  };
  GraphEntry graphs[8];
  int n_graphs = 0;
  uint64_t use_clock = 0;
};

}  // namespace ehc
