// kernels_build.cu -- once-per-MD-step kernels: fixed-point binning, cell
// sort, neighbour list, local lattice temperature, deterministic reductions.
//
// Neighbour criterion (Sec. 2, lattice-temperature definition and the user
// cutoff of Sec. 2.1): j != i with |x_j - x_i| <= r_c, evaluated exactly on a
// 2^-20 Angstrom integer grid with the minimum image on periodic axes.  The
// cell width is >= r_c, so all neighbours lie in the 3x3x3 block of cells
// around an atom's own cell.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr double kKB = 8.617333262e-5;          // eV/K (CODATA 2018)
constexpr double kMVV = 1.66053906660e-27 * 1.0e10 / 1.602176634e-19;  // amu (A/fs)^2 -> eV

// floor(v nc / L) for 0 <= v < L < 2^31 and nc < 2^20 without a 64-bit
// division: a single-precision estimate (relative error below 2^-21, so within
// one of the quotient) corrected by exact 64-bit products
__device__ __forceinline__ int32_t cell_of(int64_t v, int32_t nc, int64_t L, float ncL) {
  const int64_t num = v * (int64_t)nc;
  int64_t c = (int64_t)__float2int_rz(__int2float_rz((int32_t)v) * ncL);
  if (c * L > num) --c;
  else if ((c + 1) * L <= num) ++c;
  return (int32_t)c;
}

__global__ void bin_kernel(const double *__restrict__ x, int64_t n, Grid g, int4 *__restrict__ q,
                           int32_t *__restrict__ count, int32_t *__restrict__ err) {
  int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n) return;
  int32_t qc[3], cc[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    // round-half-even(x 2^20), the oracle's llrint, on the integer pipes
    long long v = rint_scaled(x[3 * o + k], 20);
    const long long L = g.Lq[k];
    if (g.per[k]) {
      // one period either side without a division; further out, the floored modulo
      if (v < 0) v += L;
      else if (v >= L) v -= L;
      if (v < 0 || v >= L) {
        v %= L;
        if (v < 0) v += L;
      }
    } else if (v < 0 || v >= L) {
      atomicOr(err, ERR_BOUNDS);
      v = v < 0 ? 0 : L - 1;
    }
    qc[k] = (int32_t)v;
    const int32_t c = cell_of(v, g.nc[k], L, (float)g.nc[k] / (float)L);
    cc[k] = c >= g.nc[k] ? g.nc[k] - 1 : c;
  }
  int32_t cell = (int32_t)(cc[0] + g.nc[0] * (cc[1] + (int64_t)g.nc[1] * cc[2]));
  q[o] = make_int4(qc[0], qc[1], qc[2], cell);
  atomicAdd(count + cell, 1);
}

// exclusive scan over ncell counts: per-block scan, scan of block sums, add.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v) {
  __shared__ int32_t wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int32_t w = (lane < nw) ? wsum[lane] : 0;
    int32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) wsum[lane] = wi - w;
  }
  __syncthreads();
  int32_t res = wsum[wid] + incl - v;
  __syncthreads();
  return res;
}

__global__ void scan_tiles(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t n,
                           int32_t *__restrict__ tile_sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int32_t v[kScanPer];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int32_t ex = block_excl_scan(s);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == blockDim.x - 1) tile_sums[blockIdx.x] = ex;
}

__global__ void scan_sums(int32_t *__restrict__ sums, int64_t nt, int32_t *__restrict__ grand) {
  // one block: sequential chunks per thread, then a block scan of the chunk totals
  const int64_t per = (nt + blockDim.x - 1) / blockDim.x;
  int64_t b = threadIdx.x * per;
  int32_t s = 0;
  for (int64_t k = 0; k < per; ++k)
    if (b + k < nt) s += sums[b + k];
  int32_t ex = block_excl_scan(s);
  for (int64_t k = 0; k < per; ++k)
    if (b + k < nt) {
      int32_t t = sums[b + k];
      sums[b + k] = ex;
      ex += t;
    }
  if (threadIdx.x == blockDim.x - 1) *grand = ex;
}

__global__ void scan_add(int32_t *__restrict__ out, int64_t n, const int32_t *__restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t add = sums[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x)
    if (base + k < n) out[base + k] += add;
}

__global__ void scatter_kernel(const int4 *__restrict__ q, int64_t n, const int32_t *__restrict__ start,
                               int32_t *__restrict__ fill, int32_t *__restrict__ perm) {
  int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n) return;
  int32_t cell = q[o].w;
  int32_t r = atomicAdd(fill + cell, 1);
  perm[start[cell] + r] = (int32_t)o;
}

// order each cell's atoms by original id (the scatter order is not deterministic)
// the atoms of each cell by original id: each atom's place in its cell is the
// number of the cell's atoms with a smaller id (a rank sort, one thread per atom,
// from the scatter's unordered runs into perm)
__global__ void rank_cells_kernel(int64_t n, const int4 *__restrict__ q, const int32_t *__restrict__ start,
                                  const int32_t *__restrict__ raw, int32_t *__restrict__ perm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t key = raw[i];
  const int32_t cell = q[key].w;
  const int32_t b = start[cell], e = start[cell + 1];
  int32_t r = 0;
  for (int32_t j = b; j < e; ++j) r += raw[j] < key ? 1 : 0;
  perm[b + r] = key;
}

// move per-atom data into the new sorted order
// velocity of sorted atom s from the caller-order array: on the 2^-48 A/fs grid
// (exact momentum sums) with |v|^2 in FP64, and the speed guard
__device__ __forceinline__ void gather_velocity(int64_t s, int64_t o, const double *__restrict__ v,
                                                VelQ *__restrict__ v_s, int32_t *__restrict__ err) {
  const double vx = v[3 * o + 0], vy = v[3 * o + 1], vz = v[3 * o + 2];
  // |v| < 256 = 2^8 per component, tested on the exponent bits
  if (!(abs_below_pow2(vx, 8) && abs_below_pow2(vy, 8) && abs_below_pow2(vz, 8))) atomicOr(err, ERR_SPEED);
  VelQ vq;
  vq.x = rint_scaled(vx, 48);   // round-half-even(v 2^48)
  vq.y = rint_scaled(vy, 48);
  vq.z = rint_scaled(vz, 48);
  vq.w = vx * vx + vy * vy + vz * vz;
  v_s[s] = vq;
}

// the velocities alone, for a build whose velocities arrive after its neighbour search
__global__ void gather_vel_kernel(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ v,
                                  VelQ *__restrict__ v_s, int32_t *__restrict__ err) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  gather_velocity(s, perm[s], v, v_s, err);
}

// v == nullptr: the velocities are gathered later by gather_vel_kernel
__global__ void gather_kernel(int64_t n, const int32_t *__restrict__ perm, const int4 *__restrict__ q,
                              const double *__restrict__ v, const int32_t *__restrict__ type_orig,
                              const int32_t *__restrict__ inv_old, int src_is_orig,
                              const double *__restrict__ T_old, const double *__restrict__ A_old,
                              int32_t *__restrict__ inv_new, int4 *__restrict__ q_s,
                              VelQ *__restrict__ v_s, int8_t *__restrict__ type_s,
                              double *__restrict__ T_new, double *__restrict__ A_new,
                              float *__restrict__ dmir0, double Tref, double invTmax,
                              const double *__restrict__ depth, float *__restrict__ srcw,
                              double *__restrict__ srcw_d, double inv_lp, int32_t *__restrict__ err) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  int32_t o = perm[s];
  q_s[s] = q[o];
  inv_new[o] = (int32_t)s;
  if (v) gather_velocity(s, o, v, v_s, err);
  int32_t ty = type_orig ? type_orig[o] : 0;
  type_s[s] = (int8_t)(ty < 0 ? 0 : (ty >= kMaxTypes ? kMaxTypes - 1 : ty));
  int64_t src = src_is_orig ? (int64_t)o : (int64_t)inv_old[o];
  double T = T_old[src];
  T_new[s] = T;
  A_new[s] = A_old[src];
  dmir0[s] = d2f_rn((T - Tref) * invTmax);
  if (depth) {   // source weights only with a laser source (nothing reads them otherwise)
    const double w = exp(-depth[o] * inv_lp);
    srcw[s] = (float)w;
    srcw_d[s] = w;
  }
}

// One thread per atom.  Candidates come from the atom's (deduplicated) neighbour
// rows and, within each row, the (deduplicated) cells cx-1, cx, cx+1.  All
// arithmetic is on the integer grid: per-axis minimum image in int32, the
// squared distance in int64, inclusive comparison with r_c^2.  Outputs:
//   nbr  [W][N] sorted indices in visit order (row, cell, sorted index)
//   pidx [W/2][ps] the same neighbours as 16-bit indices into the row tile (the
//        concatenation of the neighbour rows), two per word; unused slots up to
//        W hold the atom's own tile index, whose pair term is exactly zero.
// FAST: every periodic axis has at least 3 cells.  Cells are at least r_c wide,
// so a pair within r_c sits in adjacent cells and its minimum image is the
// image of that cell offset: the shift (0 or +-L) is fixed per neighbour row
// (y, z) and per cell (x), and the per-pair test is branch-free (the unsigned
// 64-bit sum of squares cannot overflow).  Otherwise each difference takes its
// minimum image separately, as in the oracle.
__device__ __forceinline__ uint32_t wrap_shift(int32_t dcell, int64_t L) {
  return dcell > 1 ? (uint32_t)(-L) : (dcell < -1 ? (uint32_t)L : 0u);
}

// the unused slots mm..W-1 of atom s (rounded up to whole words) hold its own
// tile index, whose pair term is exactly zero: whole 32-bit words after an odd
// slot, coalesced over consecutive atoms
__device__ __forceinline__ void pad_pidx(uint16_t *__restrict__ pidx16, int64_t ps, int32_t s, int32_t mm,
                                         int32_t W, uint16_t self) {
  int32_t k = mm;
  if (k & 1) {
    pidx16[((int64_t)(k >> 1) * ps + s) * 2 + 1] = self;
    ++k;
  }
  uint32_t *pw = reinterpret_cast<uint32_t *>(pidx16);
  const uint32_t two = (uint32_t)self | ((uint32_t)self << 16);
  for (int32_t w = k >> 1; w < (W + 1) >> 1; ++w) pw[(int64_t)w * ps + s] = two;
}

// The search of one atom s (the visit order and outputs described above);
// returns its neighbour count (before truncation to W), the 4-word aligned end
// of its row tile and the length of its own row.
template <bool FAST, bool WEIGHTS>
__device__ __forceinline__ int3 search_atom(int32_t s, int32_t n, const Grid &g, const int4 *__restrict__ q_s,
                                            const int32_t *__restrict__ start, const int32_t *__restrict__ row_nbr,
                                            int32_t W, int32_t *__restrict__ nbr, uint16_t *__restrict__ pidx16,
                                            int64_t ps, uint8_t *__restrict__ cnt, int32_t *__restrict__ err,
                                            float *__restrict__ wgt, float wn, double *__restrict__ wgt_d,
                                            double2 wq) {
  const int4 qi = q_s[s];
  const int32_t ncx = g.nc[0];
  const int32_t cx = qi.w % ncx;
  const int32_t R = qi.w / ncx;
  int32_t xo[3] = {0, 0, 0};
  int nx = 0;
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    int32_t c = cx + d;
    if (g.per[0]) {
      if (c < 0) c += ncx;
      if (c >= ncx) c -= ncx;
    } else if (c < 0 || c >= ncx) {
      continue;
    }
    bool dup = false;
    for (int m = 0; m < nx; ++m) dup |= (xo[m] == c);
    if (!dup) xo[nx++] = c;
  }
  // FAST: the cells xo[] in visit order form at most two runs of consecutive
  // cell indices (the second after a periodic wrap), i.e. at most two
  // contiguous atom ranges per neighbour row, each with one x image shift
  int nseg = 0;
  int32_t seg_lo[2] = {0, 0}, seg_hi[2] = {-1, -1};
  uint32_t seg_shift[2] = {0u, 0u};
  if (FAST) {
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
      if (ix >= nx) break;
      const int32_t c = xo[ix];
      if (ix > 0 && c == xo[ix - 1] + 1) {
        if (nseg == 1) seg_hi[0] = c;
        else seg_hi[1] = c;
      } else {
        const uint32_t sh = wrap_shift(c - cx, g.Lq[0]);
        if (nseg == 0) {
          seg_lo[0] = seg_hi[0] = c;
          seg_shift[0] = sh;
        } else {
          seg_lo[1] = seg_hi[1] = c;
          seg_shift[1] = sh;
        }
        ++nseg;
      }
    }
  }
  const int32_t L0 = (int32_t)g.Lq[0], L1 = (int32_t)g.Lq[1], L2 = (int32_t)g.Lq[2];
  const int32_t h0 = L0 >> 1, h1 = L1 >> 1, h2 = L2 >> 1;
  const int32_t rcq = (int32_t)g.rcq;
  const int64_t rc2 = g.rcq * g.rcq;
  int32_t m = 0;
  int32_t prefix = 0;   // tile offset of the current neighbour row
  int32_t tend = 0;     // end of the tile so far
  int32_t self_local = 0;
  int32_t own_len = 0;
  for (int r = 0; r < kRowNbr; ++r) {
    const int32_t R2 = row_nbr[(int64_t)R * kRowNbr + r];
    if (R2 < 0) break;
    const int32_t rs = start[(int64_t)R2 * ncx];
    const int32_t re = start[(int64_t)R2 * ncx + ncx];
    // row placement in the tile: after the previous row rounded up to 4 words,
    // congruent to its first index modulo 4, so that the 16-byte aligned
    // superset of every row lands on free words
    prefix = ((tend + 3) & ~3) + (rs & 3);
    if (R2 == R) {
      self_local = prefix + (s - rs);
      own_len = re - rs;
    }
    if (FAST) {
      const int32_t ny = g.nc[1];
      // dx = qj.x + ox (mod 2^32) is the minimum-image difference for every pair within r_c
      const uint32_t oy = wrap_shift(R2 % ny - R % ny, g.Lq[1]) - (uint32_t)qi.y;
      const uint32_t oz = wrap_shift(R2 / ny - R / ny, g.Lq[2]) - (uint32_t)qi.z;
      const uint64_t rc2u = (uint64_t)rc2;
      const int32_t *rowst = start + (int64_t)R2 * ncx;
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        if (sg >= nseg) break;
        const uint32_t ox = seg_shift[sg] - (uint32_t)qi.x;
        const int32_t t1 = rowst[seg_hi[sg] + 1];
        for (int32_t t = rowst[seg_lo[sg]]; t < t1; ++t) {
          const int4 qj = q_s[t];
          const int32_t dx = (int32_t)((uint32_t)qj.x + ox);
          const int32_t dy = (int32_t)((uint32_t)qj.y + oy);
          const int32_t dz = (int32_t)((uint32_t)qj.z + oz);
          const uint64_t d2 = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) +
                              (uint64_t)((int64_t)dz * dz);
          if (d2 <= rc2u && t != s) {
            if (m < W) {
              nbr[(int64_t)m * n + s] = t;
              pidx16[((int64_t)(m >> 1) * ps + s) * 2 + (m & 1)] = (uint16_t)(prefix + (t - rs));
              if (WEIGHTS) {
                wgt[(int64_t)m * n + s] = __fdiv_rn(wn, __ull2float_rn(d2 > 0 ? (uint64_t)d2 : 1ull));
                if (wgt_d) wgt_d[(int64_t)m * n + s] = wq.x / (wq.y * (double)(d2 > 0 ? (uint64_t)d2 : 1ull));
              }
            }
            ++m;
          }
        }
      }
    } else {
      for (int ix = 0; ix < nx; ++ix) {
        const int32_t cell = R2 * ncx + xo[ix];
        const int32_t t1 = start[cell + 1];
        for (int32_t t = start[cell]; t < t1; ++t) {
          if (t == s) continue;
          const int4 qj = q_s[t];
          int32_t dx = qj.x - qi.x;
          if (g.per[0]) dx = dx > h0 ? dx - L0 : (dx < -h0 ? dx + L0 : dx);
          if (dx > rcq || dx < -rcq) continue;
          int32_t dy = qj.y - qi.y;
          if (g.per[1]) dy = dy > h1 ? dy - L1 : (dy < -h1 ? dy + L1 : dy);
          if (dy > rcq || dy < -rcq) continue;
          int32_t dz = qj.z - qi.z;
          if (g.per[2]) dz = dz > h2 ? dz - L2 : (dz < -h2 ? dz + L2 : dz);
          if (dz > rcq || dz < -rcq) continue;
          const int64_t d2 = (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
          if (d2 <= rc2) {
            if (m < W) {
              nbr[(int64_t)m * n + s] = t;
              pidx16[((int64_t)(m >> 1) * ps + s) * 2 + (m & 1)] = (uint16_t)(prefix + (t - rs));
              if (WEIGHTS) {
                wgt[(int64_t)m * n + s] = __fdiv_rn(wn, __ull2float_rn(d2 > 0 ? (uint64_t)d2 : 1ull));
                if (wgt_d) wgt_d[(int64_t)m * n + s] = wq.x / (wq.y * (double)(d2 > 0 ? (uint64_t)d2 : 1ull));
              }
            }
            ++m;
          }
        }
      }
    }
    tend = prefix + (re - rs);
  }
  if (m > W) atomicOr(err, ERR_NBR_OVERFLOW);
  const int32_t mm = m < W ? m : W;
  pad_pidx(pidx16, ps, s, mm, W, (uint16_t)self_local);
  cnt[s] = (uint8_t)mm;
  return make_int3(m, (tend + 3) & ~3, own_len);
}

template <bool FAST, bool WEIGHTS>
__global__ void __launch_bounds__(128) neighbor_kernel(int32_t n, Grid g, const int4 *__restrict__ q_s,
                                                       const int32_t *__restrict__ start,
                                                       const int32_t *__restrict__ row_nbr, int32_t W,
                                                       int32_t *__restrict__ nbr, uint16_t *__restrict__ pidx16,
                                                       int64_t ps, uint8_t *__restrict__ cnt,
                                                       int32_t *__restrict__ maxcnt, int32_t *__restrict__ maxstaged,
                                                       int32_t *__restrict__ maxrow, int32_t *__restrict__ err,
                                                       float *__restrict__ wgt, float wn,
                                                       double *__restrict__ wgt_d, double2 wq) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int3 r = search_atom<FAST, WEIGHTS>(s, n, g, q_s, start, row_nbr, W, nbr, pidx16, ps, cnt, err, wgt, wn,
                                            wgt_d, wq);
  // one atomic per warp for each of the three maxima
  const unsigned act = __activemask();
  const int32_t wm = __reduce_max_sync(act, r.x);
  const int32_t ws = __reduce_max_sync(act, r.y);
  const int32_t wr = __reduce_max_sync(act, r.z);
  if ((threadIdx.x & 31) == (__ffs(act) - 1)) {
    atomicMax(maxcnt, wm);
    atomicMax(maxstaged, ws);
    atomicMax(maxrow, wr);
  }
}

// The one-type lattice temperature of atom s from its sums over S = {s} + its c
// neighbours (Sec. 2): int64 momentum sums q of the 2^-48 grid velocities and the
// 128-bit fixed-point sum (Wh, Wl) of |v|^2 on the 2^-96 grid;
// n sum |v|^2 - |sum v|^2 = n sum |v - v_com|^2 exactly, rounded once.
__device__ __forceinline__ void lattice_finish(int64_t s, const VelQ &vi, long long qx, long long qy, long long qz,
                                               unsigned long long Wh, unsigned long long Wl, int c,
                                               double m0, const RecipTab &rt, double eps_ke, double Tref,
                                               double *__restrict__ Tl_d, float *__restrict__ Tl_f,
                                               float *__restrict__ uTl) {
  const unsigned __int128 W = ((unsigned __int128)Wh << 64) | Wl;
  const __int128 S2 = (__int128)qx * qx + (__int128)qy * qy + (__int128)qz * qz;
  // D >= 0 up to the roundings of |v|^2 and of the grid (a set moving as one): not below 0
  __int128 D = (__int128)(c + 1) * (__int128)W - S2;
  if (D < 0) D = 0;
  // T = D 2^-96 (m / 2) kMVV / (c + 1) / ((3/2) k_B dof): one coefficient per count
  double T = i128_to_double(D) * rt.coefT[c];
  const double Ks = 0.5 * m0 * vi.w * kMVV;
  const bool chi = Ks >= eps_ke;
  if (!chi) T = -1.0;
  Tl_d[s] = T;
  Tl_f[s] = d2f_rn(T);
  uTl[s] = chi ? d2f_rn(Tref - T) : __int_as_float(0x7fc00000);
}

// ---- neighbour lists from a candidate list with a skin (cells >= r_c + skin) ----
// The candidates of an atom are the atoms within r_v = r_c + skin of it when the
// candidate list was built: original ids in the visit order of that build, atom-
// major [N][Wc] by original id (one atom's list is contiguous, so a build reads
// about as many DRAM sectors as it uses).
// While no atom has moved more than skin / 2 on the grid since then, every pair
// within r_c is among them, and the list of the MD step is the candidates that
// pass the exact integer test with the current positions: the same set, and
// written in the same order, as the full cell search (row, cell run, sorted
// index).  The check below sets *flag when an atom moved further (or the list
// is new); the candidate kernel then rebuilds the list first.

__device__ __forceinline__ int32_t wrap_d(int32_t d, int32_t L, int32_t h, int per) {
  return per ? (d > h ? d - L : (d < -h ? d + L : d)) : d;
}

// *flag |= 1 if some atom moved more than skin / 2 since the candidate build
__global__ void skin_check_kernel(int32_t n, Grid g, const int4 *__restrict__ q, const int4 *__restrict__ q_ref,
                                  int64_t half2, int32_t *__restrict__ flag) {
  const int32_t o = blockIdx.x * blockDim.x + threadIdx.x;
  bool far = false;
  if (o < n) {
    const int4 a = q[o], b = q_ref[o];
    const int32_t L0 = (int32_t)g.Lq[0], L1 = (int32_t)g.Lq[1], L2 = (int32_t)g.Lq[2];
    const int64_t dx = wrap_d(a.x - b.x, L0, L0 >> 1, g.per[0]);
    const int64_t dy = wrap_d(a.y - b.y, L1, L1 >> 1, g.per[1]);
    const int64_t dz = wrap_d(a.z - b.z, L2, L2 >> 1, g.per[2]);
    far = dx * dx + dy * dy + dz * dz > half2;
  }
  if (__any_sync(0xffffffffu, far) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// Candidate list (only when *flag is set): the full cell search with r_v, one
// thread per sorted atom, candidates as original ids in visit order, atom-major
// by original id; the positions of the build go to q_ref.  FAST grids only (>= 3 cells per periodic
// axis, cells at least r_v wide).
__global__ void __launch_bounds__(128) cand_kernel(int32_t n, Grid g, int64_t rv2, const int4 *__restrict__ q_s,
                                                   const int32_t *__restrict__ perm, const int32_t *__restrict__ start,
                                                   const int32_t *__restrict__ row_nbr, int32_t Wc,
                                                   int32_t *__restrict__ cand, uint8_t *__restrict__ ccnt,
                                                   const int4 *__restrict__ q_orig, int4 *__restrict__ q_ref,
                                                   const int32_t *__restrict__ flag, int32_t *__restrict__ err) {
  if (*flag == 0) return;
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int4 qi = q_s[s];
  const int32_t o = perm[s];
  q_ref[o] = q_orig[o];
  const int32_t ncx = g.nc[0], ny = g.nc[1];
  const int32_t cx = qi.w % ncx, R = qi.w / ncx;
  int32_t m = 0;
  for (int r = 0; r < kRowNbr; ++r) {
    const int32_t R2 = row_nbr[(int64_t)R * kRowNbr + r];
    if (R2 < 0) break;
    const uint32_t oy = wrap_shift(R2 % ny - R % ny, g.Lq[1]) - (uint32_t)qi.y;
    const uint32_t oz = wrap_shift(R2 / ny - R / ny, g.Lq[2]) - (uint32_t)qi.z;
    const int32_t *rowst = start + (int64_t)R2 * ncx;
    for (int d = -1; d <= 1; ++d) {
      int32_t c = cx + d;
      if (g.per[0]) c = c < 0 ? c + ncx : (c >= ncx ? c - ncx : c);
      else if (c < 0 || c >= ncx) continue;
      const uint32_t ox = wrap_shift(c - cx, g.Lq[0]) - (uint32_t)qi.x;
      for (int32_t t = rowst[c]; t < rowst[c + 1]; ++t) {
        const int4 qj = q_s[t];
        const int32_t dx = (int32_t)((uint32_t)qj.x + ox);
        const int32_t dy = (int32_t)((uint32_t)qj.y + oy);
        const int32_t dz = (int32_t)((uint32_t)qj.z + oz);
        const uint64_t d2 = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) +
                            (uint64_t)((int64_t)dz * dz);
        if (d2 <= (uint64_t)rv2 && t != s) {
          if (m < Wc) cand[(int64_t)o * Wc + m] = perm[t];
          ++m;
        }
      }
    }
  }
  if (m > Wc) atomicOr(err, ERR_NBR_OVERFLOW);
  ccnt[o] = (uint8_t)(m < Wc ? m : Wc);
}

// The list of the MD step from the candidates: the same outputs as
// neighbor_kernel<true, false> (nbr, pidx, cnt, maxima), in its visit order (row,
// cell run, sorted index).  The candidates are kept in the visit order of the
// last build that sorted them, and the hits come out in that order unless a
// candidate changed cell since; each hit's visit key (row place, cell run,
// sorted index) is checked against the previous one as it is written.  An atom
// whose keys do not rise sorts its candidate list by the current keys (an
// insertion sort in local memory, rare: an atom that crosses a cell face
// unsorts the lists of its ~20 candidates once), writes it back for the next
// builds and writes its hits again in that order.  Every list is exactly the
// full search's.
constexpr int kFilterBatch = 2;     // candidates whose three dependent loads are in flight together
constexpr int kFilterThreads = 128;

// floor(x / d) for 0 <= x < 2^31 and d >= 1, with mg = floor(2^32 / d) (d > 1; any
// value for d = 1): the high product is the quotient or one less
__device__ __forceinline__ int32_t udiv_mg(int32_t x, int32_t d, uint32_t mg) {
  if (d == 1) return x;
  int32_t q = (int32_t)__umulhi((uint32_t)x, mg);
  if (x - q * d >= d) ++q;
  return q;
}

// a cell-index difference on a periodic axis of n cells as the offset in {-1, 0, 1}
// of adjacent cells (anything else: outside)
__device__ __forceinline__ int32_t wrap_off(int32_t d, int32_t n, int per) {
  if (per) d = d > 1 ? d - n : (d < -1 ? d + n : d);
  return d;
}

template <typename T>
__device__ __forceinline__ T sel3(const T *v, int32_t d) {   // v[d + 1] for d in {-1, 0, 1}
  return d < 0 ? v[0] : (d > 0 ? v[2] : v[1]);
}

// The atom's view of its 27 cells: per axis offset (-1, 0, 1) the image shift
// minus its own coordinate, the x offset's cell run, and per row place the tile
// base (row placement as neighbor_kernel)
struct FilterView {
  int32_t cx, cy, cz, dy_lo, dz_lo, nyc;
  uint32_t sx[3], sy[3], sz[3];
  int32_t run[3];
  const int32_t *base;   // the rows' tile bases in shared memory, row place r at base[r * kFilterThreads]
};

// the visit class 2 r + run of a candidate in cell cw (false: outside the 27 cells),
// its shifts and tile base
__device__ __forceinline__ bool classify(const FilterView &fv, const Grid &g, uint32_t mgx, uint32_t mgy,
                                         int32_t cw, int &cls, uint32_t &ox, uint32_t &oy, uint32_t &oz,
                                         int32_t &bs) {
  const int32_t ncx = g.nc[0], ny = g.nc[1];
  const int32_t R2 = udiv_mg(cw, ncx, mgx);
  const int32_t cz = udiv_mg(R2, ny, mgy);
  const int32_t dx = wrap_off(cw - R2 * ncx - fv.cx, ncx, g.per[0]);
  const int32_t dy = wrap_off(R2 - cz * ny - fv.cy, ny, g.per[1]);
  const int32_t dz = wrap_off(cz - fv.cz, g.nc[2], g.per[2]);
  if ((uint32_t)(dx + 1) > 2u || (uint32_t)(dy + 1) > 2u || (uint32_t)(dz + 1) > 2u) return false;
  const int r = (dz - fv.dz_lo) * fv.nyc + (dy - fv.dy_lo);
  ox = sel3(fv.sx, dx);
  oy = sel3(fv.sy, dy);
  oz = sel3(fv.sz, dz);
  bs = fv.base[r * kFilterThreads];
  cls = 2 * r + sel3(fv.run, dx);
  return true;
}

// The list of the MD step from the candidates: the same outputs as
// neighbor_kernel<true, false> (nbr, pidx, cnt, maxima), in its visit order (row,
// cell run, sorted index).  The candidates are kept in the visit order of the
// last build that sorted them, and the hits come out in that order unless a
// candidate changed cell since; each hit's visit key (row place, cell run,
// sorted index) is checked against the previous one as it is written.  An atom
// whose keys do not rise sorts its candidate list by the current keys (an
// insertion sort in local memory, rare: an atom that crosses a cell face
// unsorts the lists of its ~20 candidates once), writes it back for the next
// builds and writes its hits again in that order.  Every list is exactly the
// full search's.  A candidate's cell offsets come from its cell index by two
// multiply-high divisions (mgx, mgy: floor(2^32 / cells) of the x and y axes).
__global__ void __launch_bounds__(kFilterThreads) filter_kernel(int32_t n, Grid g, uint32_t mgx, uint32_t mgy,
                                                     const int4 *__restrict__ q_s,
                                                     const int32_t *__restrict__ perm, const int32_t *__restrict__ inv,
                                                     const int32_t *__restrict__ start,
                                                     const int32_t *__restrict__ row_nbr, int32_t W, int32_t Wc,
                                                     int32_t *__restrict__ cand, uint8_t *__restrict__ ccnt,
                                                     int32_t *__restrict__ nbr, uint16_t *__restrict__ pidx16,
                                                     int64_t ps, uint8_t *__restrict__ cnt,
                                                     int32_t *__restrict__ maxcnt, int32_t *__restrict__ maxstaged,
                                                     int32_t *__restrict__ maxrow, int32_t *__restrict__ err) {
  __shared__ int32_t sbase[kRowNbr * kFilterThreads];   // each thread's column: its rows' tile bases
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int4 qi = q_s[s];
  const int32_t o = perm[s];
  const int c = ccnt[o];
  int32_t *cl = cand + (int64_t)o * Wc;
  const int32_t ncx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
  FilterView fv;
  int32_t *mybase = sbase + threadIdx.x;
  fv.base = mybase;
  const int32_t R = udiv_mg(qi.w, ncx, mgx);
  fv.cx = qi.w - R * ncx;
  fv.cz = udiv_mg(R, ny, mgy);
  fv.cy = R - fv.cz * ny;
  fv.dy_lo = (g.per[1] || fv.cy > 0) ? -1 : 0;
  fv.dz_lo = (g.per[2] || fv.cz > 0) ? -1 : 0;
  fv.nyc = ((g.per[1] || fv.cy < ny - 1) ? 1 : 0) - fv.dy_lo + 1;
  // per offset: the wrapped neighbour cell's image shift (wrap_shift of the raw
  // cell difference, as the full search), minus the atom's own coordinate
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    int32_t xw = fv.cx + d, yw = fv.cy + d, zw = fv.cz + d;
    if (g.per[0]) xw = xw < 0 ? xw + ncx : (xw >= ncx ? xw - ncx : xw);
    if (g.per[1]) yw = yw < 0 ? yw + ny : (yw >= ny ? yw - ny : yw);
    if (g.per[2]) zw = zw < 0 ? zw + nz : (zw >= nz ? zw - nz : zw);
    fv.sx[d + 1] = wrap_shift(xw - fv.cx, g.Lq[0]) - (uint32_t)qi.x;
    fv.sy[d + 1] = wrap_shift(yw - fv.cy, g.Lq[1]) - (uint32_t)qi.y;
    fv.sz[d + 1] = wrap_shift(zw - fv.cz, g.Lq[2]) - (uint32_t)qi.z;
  }
  // x runs in visit order (cx-1, cx, cx+1; a run restarts where the cells wrap)
  fv.run[0] = 0;
  fv.run[1] = (g.per[0] && fv.cx == 0) ? 1 : 0;
  fv.run[2] = fv.run[1] + ((g.per[0] && fv.cx == ncx - 1) ? 1 : 0);
  if (!g.per[0] && fv.cx == 0) {   // no cell at -1: the runs start at the own cell
    fv.run[1] = 0;
    fv.run[2] = 0;
  }
  int32_t tend = 0, self_local = 0, own_len = 0;
  bool rows_done = false;
#pragma unroll
  for (int r = 0; r < kRowNbr; ++r) {
    mybase[r * kFilterThreads] = 0;
    const int32_t R2 = rows_done ? -1 : row_nbr[(int64_t)R * kRowNbr + r];
    if (R2 < 0) {
      rows_done = true;
      continue;
    }
    const int32_t a = start[(int64_t)R2 * ncx], b = start[(int64_t)R2 * ncx + ncx];
    const int32_t pr = ((tend + 3) & ~3) + (a & 3);
    mybase[r * kFilterThreads] = pr - a;
    if (R2 == R) {
      self_local = pr + (s - a);
      own_len = b - a;
    }
    tend = pr + (b - a);
  }
  const uint64_t rc2u = (uint64_t)(g.rcq * g.rcq);
  int m = 0;
  uint64_t last = 0;
  bool ordered = true;
  for (int k0 = 0; k0 < c; k0 += kFilterBatch) {
    int32_t t[kFilterBatch];
    int4 qj[kFilterBatch];
#pragma unroll
    for (int u = 0; u < kFilterBatch; ++u) t[u] = k0 + u < c ? cl[k0 + u] : -1;
#pragma unroll
    for (int u = 0; u < kFilterBatch; ++u) t[u] = t[u] >= 0 ? inv[t[u]] : -1;
#pragma unroll
    for (int u = 0; u < kFilterBatch; ++u) qj[u] = q_s[t[u] >= 0 ? t[u] : s];
#pragma unroll
    for (int u = 0; u < kFilterBatch; ++u) {
      if (t[u] < 0 || t[u] == s) continue;
      int cls;
      uint32_t ox, oy, oz;
      int32_t bs;
      if (!classify(fv, g, mgx, mgy, qj[u].w, cls, ox, oy, oz, bs)) {
        ordered = false;   // a candidate left the 27 cells: dropped at the re-sort
        continue;
      }
      const int32_t dx = (int32_t)((uint32_t)qj[u].x + ox);
      const int32_t dy = (int32_t)((uint32_t)qj[u].y + oy);
      const int32_t dz = (int32_t)((uint32_t)qj[u].z + oz);
      const uint64_t d2 =
          (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) + (uint64_t)((int64_t)dz * dz);
      if (d2 > rc2u) continue;
      const uint64_t key = ((uint64_t)cls << 32) | (uint32_t)t[u];
      if (m > 0 && key <= last) ordered = false;
      last = key;
      if (m < W) {
        nbr[(int64_t)m * n + s] = t[u];
        pidx16[((int64_t)(m >> 1) * ps + s) * 2 + (m & 1)] = (uint16_t)(bs + t[u]);
      }
      ++m;
    }
  }
  if (!ordered) {
    // sort the candidates by their current visit keys (those outside the 27 cells
    // dropped), write the list back, and the hits again in that order
    uint64_t key[kCandWidth];
    int32_t id[kCandWidth];
    int nc = 0;
    for (int k = 0; k < c; ++k) {
      const int32_t idk = cl[k];
      const int32_t tk = inv[idk];
      int cls;
      uint32_t ox, oy, oz;
      int32_t bs;
      if (tk == s || !classify(fv, g, mgx, mgy, q_s[tk].w, cls, ox, oy, oz, bs)) continue;
      const uint64_t kk = ((uint64_t)cls << 32) | (uint32_t)tk;
      int p = nc;
      while (p > 0 && key[p - 1] > kk) {
        key[p] = key[p - 1];
        id[p] = id[p - 1];
        --p;
      }
      key[p] = kk;
      id[p] = idk;
      ++nc;
    }
    m = 0;
    for (int k = 0; k < nc; ++k) {
      cl[k] = id[k];
      const int32_t tk = (int32_t)(uint32_t)key[k];
      const int4 qk = q_s[tk];
      int cls;
      uint32_t ox = 0u, oy = 0u, oz = 0u;
      int32_t bs = 0;
      classify(fv, g, mgx, mgy, qk.w, cls, ox, oy, oz, bs);
      const int32_t dx = (int32_t)((uint32_t)qk.x + ox);
      const int32_t dy = (int32_t)((uint32_t)qk.y + oy);
      const int32_t dz = (int32_t)((uint32_t)qk.z + oz);
      const uint64_t d2 =
          (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) + (uint64_t)((int64_t)dz * dz);
      if (d2 > rc2u) continue;
      if (m < W) {
        nbr[(int64_t)m * n + s] = tk;
        pidx16[((int64_t)(m >> 1) * ps + s) * 2 + (m & 1)] = (uint16_t)(bs + tk);
      }
      ++m;
    }
    // candidates that left the 27 cells are gone from the list written back
    if (nc != c) ccnt[o] = (uint8_t)nc;
  }
  if (m > W) atomicOr(err, ERR_NBR_OVERFLOW);
  const int32_t mm = m < W ? m : W;
  pad_pidx(pidx16, ps, s, mm, W, (uint16_t)self_local);
  cnt[s] = (uint8_t)mm;
  const unsigned act = __activemask();
  const int32_t wm = __reduce_max_sync(act, m);
  const int32_t ws = __reduce_max_sync(act, (tend + 3) & ~3);
  const int32_t wr = __reduce_max_sync(act, own_len);
  if ((threadIdx.x & 31) == (__ffs(act) - 1)) {
    atomicMax(maxcnt, wm);
    atomicMax(maxstaged, ws);
    atomicMax(maxrow, wr);
  }
}

// Sec. 2: T_i^lat = sum_S (1/2) m |v - v_com|^2 / ((3/2) k_B N_j) over S = {i} + neighbours.
// With M = sum m, P = sum m v, W = sum m |v|^2:  sum (1/2) m |v - v_com|^2 = (W - |P|^2 / M) / 2.
// One atom type: M = m N_j, P = m sum v with sum v exact on the 2^-48 grid
// (int64), W = m sum |v|^2 (one FP64 addition per neighbour).  Several types:
// FP64 sums of m v and m |v|^2.
template <bool ONE_TYPE>
__global__ void lattice_temp_kernel(int64_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt,
                                    const VelQ *__restrict__ v_s, const int8_t *__restrict__ type_s,
                                    MassTable mt, RecipTab rt, int dof_mode, double eps_ke, double Tref,
                                    double *__restrict__ Tl_d, float *__restrict__ Tl_f, float *__restrict__ uTl,
                                    int32_t *__restrict__ err) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int c = cnt[s];
  const VelQ vi = v_s[s];
  double T;
  if (ONE_TYPE) {
    // n sum_S |v|^2 - |sum_S v|^2 = n sum_S |v - v_com|^2 exactly on the 2^-96 grid:
    // int64 momentum sums of the fixed-point velocities and a 128-bit fixed-point
    // sum of the FP64 |v|^2 (no cancellation, no FP64 pipe in the loop)
    long long qx = vi.x, qy = vi.y, qz = vi.z;
    unsigned long long Wh = 0, Wl = 0;
    fix96_add(Wh, Wl, vi.w);
    // neighbours four at a time, software-pipelined: the next four indices are
    // loaded while this four's velocities are summed (two gathers in flight)
    int k = 0;
    int32_t tn[4];
    if (c >= 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) tn[u] = (int32_t)checked_index(nbr[(int64_t)u * n + s], (uint32_t)n, err);
    }
    for (; k + 4 <= c; k += 4) {
      VelQ vj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) vj[u] = v_s[tn[u]];
      if (k + 8 <= c) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          tn[u] = (int32_t)checked_index(nbr[(int64_t)(k + 4 + u) * n + s], (uint32_t)n, err);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        qx += vj[u].x;
        qy += vj[u].y;
        qz += vj[u].z;
        fix96_add(Wh, Wl, vj[u].w);
      }
    }
    for (; k < c; ++k) {
      const VelQ vj = v_s[checked_index(nbr[(int64_t)k * n + s], (uint32_t)n, err)];
      qx += vj.x;
      qy += vj.y;
      qz += vj.z;
      fix96_add(Wh, Wl, vj.w);
    }
    lattice_finish(s, vi, qx, qy, qz, Wh, Wl, c, mt.m[0], rt, eps_ke, Tref, Tl_d, Tl_f, uTl);
    return;
  } else {
    const double mi = mt.m[type_s[s]];
    double M = mi;
    double px = mi * ((double)vi.x * kVelUnit);
    double py = mi * ((double)vi.y * kVelUnit);
    double pz = mi * ((double)vi.z * kVelUnit);
    double W = mi * vi.w;
    for (int k = 0; k < c; ++k) {
      const int32_t t = checked_index(nbr[(int64_t)k * n + s], (uint32_t)n, err);
      const VelQ vj = v_s[t];
      const double mj = mt.m[type_s[t]];
      M += mj;
      px += mj * ((double)vj.x * kVelUnit);
      py += mj * ((double)vj.y * kVelUnit);
      pz += mj * ((double)vj.z * kVelUnit);
      W += mj * vj.w;
    }
    const double ke = fmax(0.5 * (W - (px * px + py * py + pz * pz) / M) * kMVV, 0.0);
    const int dof = (dof_mode == 1) ? c : c + 1;
    T = dof > 0 ? ke * rt.inv_dof[dof] : 0.0;
  }
  const double Ks = 0.5 * mt.m[ONE_TYPE ? 0 : type_s[s]] * vi.w * kMVV;
  const bool chi = Ks >= eps_ke;
  if (!chi) T = -1.0;
  Tl_d[s] = T;
  Tl_f[s] = (float)T;
  uTl[s] = chi ? (float)(Tref - T) : __int_as_float(0x7fc00000);
}

// Deterministic block reduction helpers: fixed thread-to-element map and a fixed
// shuffle tree, so sums are identical run to run.
__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

__device__ __forceinline__ double block_max(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = -1e300;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : -1e300;
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  return r;
}

// electronic energy per unit volume: int_0^T min(gamma T', cap) dT' [J m^-3]
__device__ __forceinline__ double ce_integral(double t, double gamma, double cap) {
  if (cap > 0.0 && gamma * t > cap) {
    const double Tc = cap / gamma;
    return 0.5 * cap * Tc + cap * (t - Tc);
  }
  return 0.5 * gamma * t * t;
}

// partial sums per block (stride kGlob): [0] sum T, [1] max T, [2] sum KE (eV),
// [3] sum srcw, [4] max(-T), [5] sum of the energy integral if gamma > 0
constexpr int kGlob = 6;
__global__ void globals_partial(int64_t n, const double *__restrict__ T, const VelQ *__restrict__ v_s,
                                const int8_t *__restrict__ type_s, MassTable mt,
                                const float *__restrict__ srcw, const double *__restrict__ srcw_d, double gamma,
                                double cap, double *__restrict__ part) {
  __shared__ double sh[32];
  double sT = 0, mT = -1e300, sK = 0, sW = 0, mN = -1e300, sE = 0;
  // the largest and smallest T on the integer pipes: bit patterns mapped to keys
  // that order like the values (NaN skipped, as fmax does); one atom type: the sum
  // of |v|^2, times m kMVV / 2 once per thread
  const bool one = mt.n_types == 1;
  long long kmax = (long long)0x8000000000000000ull, kmin = 0x7fffffffffffffffll;
  bool any = false;
  double sw = 0.0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    double t = T[s];
    sT += t;
    const long long b = __double_as_longlong(t);
    if ((b & 0x7fffffffffffffffll) <= 0x7ff0000000000000ll) {
      const long long k = b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
      kmax = k > kmax ? k : kmax;
      kmin = k < kmin ? k : kmin;
      any = true;
    }
    if (gamma > 0.0) sE += ce_integral(t, gamma, cap);
    if (v_s) {
      if (one) sw += v_s[s].w;
      else sK += 0.5 * mt.m[type_s[s]] * v_s[s].w * kMVV;
    }
    if (srcw_d) sW += srcw_d[s];
    else if (srcw) sW += (double)srcw[s];
  }
  if (any) {
    mT = __longlong_as_double(kmax >= 0 ? kmax : (kmax ^ 0x7fffffffffffffffll));
    mN = -__longlong_as_double(kmin >= 0 ? kmin : (kmin ^ 0x7fffffffffffffffll));
  }
  if (v_s && one) sK = 0.5 * mt.m[0] * sw * kMVV;
  double r0 = block_sum(sT, sh);
  double r1 = block_max(mT, sh);
  double r2 = block_sum(sK, sh);
  double r3 = block_sum(sW, sh);
  double r4 = block_max(mN, sh);
  double r5 = block_sum(sE, sh);
  if (threadIdx.x == 0) {
    double *o = part + (int64_t)blockIdx.x * kGlob;
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
    o[3] = r3;
    o[4] = r4;
    o[5] = r5;
  }
}

__global__ void globals_final(int nb, const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double sh[32];
  double sT = 0, mT = -1e300, sK = 0, sW = 0, mN = -1e300, sE = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double *q = part + (int64_t)b * kGlob;
    sT += q[0];
    mT = fmax(mT, q[1]);
    sK += q[2];
    sW += q[3];
    mN = fmax(mN, q[4]);
    sE += q[5];
  }
  double r0 = block_sum(sT, sh);
  double r1 = block_max(mT, sh);
  double r2 = block_sum(sK, sh);
  double r3 = block_sum(sW, sh);
  double r4 = block_max(mN, sh);
  double r5 = block_sum(sE, sh);
  if (threadIdx.x == 0) {
    out[0] = r0;
    out[1] = r1;
    out[2] = r2;
    out[3] = r3;
    out[4] = r4;
    out[5] = r5;
  }
}

// initial electronic energy: partials [0] sum T, [1] max T, [2] sum of the
// energy integral [J m^-3], [3] 0, [4] max(-T), [5] the integral again
__global__ void seed_partial(int64_t n, const double *__restrict__ T, double gamma, double cap,
                             double *__restrict__ part) {
  __shared__ double sh[32];
  double sT = 0, mT = -1e300, sE = 0, mN = -1e300;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const double t = T[s];
    sT += t;
    mT = fmax(mT, t);
    mN = fmax(mN, -t);
    sE += ce_integral(t, gamma, cap);
  }
  double r0 = block_sum(sT, sh);
  double r1 = block_max(mT, sh);
  double r2 = block_sum(sE, sh);
  double r4 = block_max(mN, sh);
  if (threadIdx.x == 0) {
    double *o = part + (int64_t)blockIdx.x * kGlob;
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
    o[3] = 0.0;
    o[4] = r4;
    o[5] = r2;
  }
}

__global__ void unpermute_kernel(int64_t n, const int32_t *__restrict__ inv, const double *__restrict__ src,
                                 double *__restrict__ dst) {
  int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n) return;
  dst[o] = inv ? src[inv[o]] : src[o];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// reciprocal tables of the lattice temperature
static RecipTab recip_table(const Ctx &c) {
  RecipTab rt;
  for (int k = 0; k < kMaxWidth + 2; ++k) {
    rt.inv_n[k] = k > 0 ? 1.0 / (double)k : 0.0;
    rt.inv_dof[k] = k > 0 ? 1.0 / (1.5 * kKB * (double)k) : 0.0;
    // one atom type: T = D 2^-96 (m / 2) kMVV / (k + 1) / ((3/2) k_B dof) for k neighbours
    const int dof = (c.p.dof_mode == 1) ? k : k + 1;
    rt.coefT[k] = dof > 0 ? std::ldexp(0.5 * c.mt.m[0] * kMVV, -96) / (double)(k + 1) / (1.5 * kKB * (double)dof)
                          : 0.0;
  }
  return rt;
}

cudaError_t launch_bin(Ctx &c, const double *x) {
  cudaMemsetAsync(c.cell_count, 0, sizeof(int32_t) * (c.g.ncell + 1), c.stream);
  if (c.n > 0) bin_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(x, c.n, c.g, c.q_orig, c.cell_count, c.err);
  // exclusive scan of the counts into cell_start[0..ncell], cell_start[ncell] = n
  const int64_t nt = (c.g.ncell + kScanTile - 1) / kScanTile;
  scan_tiles<<<(unsigned)nt, kScanThreads, 0, c.stream>>>(c.cell_count, c.cell_start, c.g.ncell, c.scan_tmp);
  scan_sums<<<1, kScanThreads, 0, c.stream>>>(c.scan_tmp, nt, c.cell_start + c.g.ncell);
  scan_add<<<(unsigned)nt, 256, 0, c.stream>>>(c.cell_start, c.g.ncell, c.scan_tmp);
  return cudaGetLastError();
}

cudaError_t launch_sort_cells(Ctx &c) {
  cudaMemsetAsync(c.cell_fill, 0, sizeof(int32_t) * c.g.ncell, c.stream);
  if (c.n > 0) {
    scatter_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(c.q_orig, c.n, c.cell_start, c.cell_fill, c.perm_raw);
    rank_cells_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(c.n, c.q_orig, c.cell_start, c.perm_raw, c.perm);
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_vel(Ctx &c, const double *v) {
  if (c.n > 0) gather_vel_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(c.n, c.perm, v, c.v_s, c.err);
  return cudaGetLastError();
}

cudaError_t launch_gather(Ctx &c, const double *v, bool src_is_orig) {
  int nxt = c.cur_inv ^ 1;
  int tn = c.tcur ^ 1;
  bool laser = c.p.laser_on && c.have_depth;
  if (c.n > 0)
    gather_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(
        c.n, c.perm, c.q_orig, v, c.type_orig, c.inv_perm[c.cur_inv], src_is_orig ? 1 : 0, c.T[c.tcur], c.A,
        c.inv_perm[nxt], c.q_s, c.v_s, c.type_s, c.T[tn], c.A_tmp, c.dmir[0], c.p.Tref_K, 1.0 / c.p.Tmax_K,
        laser ? c.depth_orig : nullptr, c.srcw, c.srcw_d, laser ? 1.0 / c.p.laser_lp_A : 0.0, c.err);
  c.cur_inv = nxt;
  c.tcur = tn;
  // A keeps its address (captured substep graphs and the tile argument table hold it)
  cudaMemcpyAsync(c.A, c.A_tmp, sizeof(double) * (c.n > 0 ? c.n : 1), cudaMemcpyDeviceToDevice, c.stream);
  c.parity = 0;
  return cudaGetLastError();
}

cudaError_t launch_neighbors(Ctx &c) {
  cudaMemsetAsync(c.maxcnt, 0, sizeof(int32_t) * 3, c.stream);
  if (c.n == 0) return cudaGetLastError();
  bool fast = true;
  for (int k = 0; k < 3; ++k) fast = fast && (!c.g.per[k] || c.g.nc[k] >= 3);
  if (c.skin_q > 0 && fast && !c.wgt && c.W <= 32) {
    // candidates with the skin: rebuilt when an atom moved more than skin / 2 (or
    // at the first build), then the exact test of this step's positions
    int32_t *flag = c.err + 4;
    if (!c.cand_valid) {
      cudaMemsetAsync(flag, 0xff, sizeof(int32_t), c.stream);
    } else {
      cudaMemsetAsync(flag, 0, sizeof(int32_t), c.stream);
      const int64_t half = c.skin_q / 2;
      skin_check_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>((int32_t)c.n, c.g, c.q_orig, c.q_ref, half * half,
                                                              flag);
    }
    const int64_t rvq = c.g.rcq + c.skin_q;
    cand_kernel<<<nblk(c.n, 128), 128, 0, c.stream>>>((int32_t)c.n, c.g, rvq * rvq, c.q_s, c.perm, c.cell_start,
                                                      c.row_nbr, kCandWidth, c.cand, c.ccnt, c.q_orig, c.q_ref, flag,
                                                      c.err);
    const uint32_t mgx = c.g.nc[0] > 1 ? (uint32_t)(4294967296ull / (uint64_t)c.g.nc[0]) : 0u;
    const uint32_t mgy = c.g.nc[1] > 1 ? (uint32_t)(4294967296ull / (uint64_t)c.g.nc[1]) : 0u;
    filter_kernel<<<nblk(c.n, kFilterThreads), kFilterThreads, 0, c.stream>>>(
        (int32_t)c.n, c.g, mgx, mgy, c.q_s, c.perm, c.inv_perm[c.cur_inv], c.cell_start, c.row_nbr, c.W, kCandWidth,
        c.cand, c.ccnt, c.nbr, reinterpret_cast<uint16_t *>(c.pidx), c.ps, c.cnt, c.maxcnt, c.maxstaged, c.maxrow,
        c.err);
    c.cand_valid = true;
    return cudaGetLastError();
  }
  // pair weights S2 / (n_shell r^2) with r^2 = d2 2^-40 A^2 (d2 on the 2^-20 A grid),
  // in single precision (as stored): d2 rounded to float, one correctly rounded division
  const double wn = c.p.rate_shell_n > 0 ? c.p.zb2_A2 * 1099511627776.0 / (double)c.p.rate_shell_n : 0.0;
  auto kern = c.wgt ? (fast ? neighbor_kernel<true, true> : neighbor_kernel<false, true>)
                    : (fast ? neighbor_kernel<true, false> : neighbor_kernel<false, false>);
  // the FP64 path's weights in FP64, as the oracle forms them: S2 2^40 / (n_shell d2)
  const double2 wq = make_double2(c.p.zb2_A2 * 1099511627776.0, (double)c.p.rate_shell_n);
  kern<<<nblk(c.n, 128), 128, 0, c.stream>>>((int32_t)c.n, c.g, c.q_s, c.cell_start, c.row_nbr, c.W, c.nbr,
                                             reinterpret_cast<uint16_t *>(c.pidx), c.ps, c.cnt, c.maxcnt,
                                             c.maxstaged, c.maxrow, c.err, c.wgt, (float)wn, c.wgt_d, wq);
  return cudaGetLastError();
}

cudaError_t launch_lattice_temperature(Ctx &c) {
  if (c.n == 0) return cudaGetLastError();
  const RecipTab rt = recip_table(c);
  if (c.mt.n_types == 1)
    lattice_temp_kernel<true><<<nblk(c.n, 256), 256, 0, c.stream>>>(c.n, c.nbr, c.cnt, c.v_s, c.type_s, c.mt, rt,
                                                                    c.p.dof_mode, c.p.eps_ke_eV, c.p.Tref_K,
                                                                    c.Tl_d, c.Tl_f, c.uTl, c.err);
  else
    lattice_temp_kernel<false><<<nblk(c.n, 256), 256, 0, c.stream>>>(c.n, c.nbr, c.cnt, c.v_s, c.type_s, c.mt, rt,
                                                                     c.p.dof_mode, c.p.eps_ke_eV, c.p.Tref_K,
                                                                     c.Tl_d, c.Tl_f, c.uTl, c.err);
  return cudaGetLastError();
}

cudaError_t launch_globals(Ctx &c) {
  const bool laser = c.p.laser_on && c.have_depth;
  globals_partial<<<kRedBlocks, kRedThreads, 0, c.stream>>>(
      c.n, c.T[c.tcur], c.v_s, c.type_s, c.mt, (laser && c.p.flux_prec == 0) ? c.srcw : nullptr,
      (laser && c.p.flux_prec == 1) ? c.srcw_d : nullptr, c.local ? c.p.gamma_Ce : 0.0, c.cap_si, c.partials);
  globals_final<<<1, kRedThreads, 0, c.stream>>>(kRedBlocks, c.partials, c.scal);
  return cudaGetLastError();
}

cudaError_t launch_ledger(Ctx &c) {
  globals_partial<<<kRedBlocks, kRedThreads, 0, c.stream>>>(c.n, c.T[c.tcur], nullptr, nullptr, c.mt, nullptr,
                                                            nullptr, c.local ? c.p.gamma_Ce : 0.0, c.cap_si,
                                                            c.partials);
  globals_final<<<1, kRedThreads, 0, c.stream>>>(kRedBlocks, c.partials, c.scal);
  return cudaGetLastError();
}

cudaError_t launch_seed(Ctx &c, double cap_SI) {
  seed_partial<<<kRedBlocks, kRedThreads, 0, c.stream>>>(c.n, c.T[c.tcur], c.p.gamma_Ce, cap_SI, c.partials);
  globals_final<<<1, kRedThreads, 0, c.stream>>>(kRedBlocks, c.partials, c.scal);
  return cudaGetLastError();
}

cudaError_t launch_unpermute(Ctx &c, const double *src_sorted, double *dst_orig, int identity) {
  if (c.n > 0)
    unpermute_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(c.n, identity ? nullptr : c.inv_perm[c.cur_inv],
                                                           src_sorted, dst_orig);
  return cudaGetLastError();
}

}  // namespace ehc
