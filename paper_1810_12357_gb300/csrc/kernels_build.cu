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

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr double kKB = 8.617333262e-5;          // eV/K (CODATA 2018)
constexpr double kMVV = 1.66053906660e-27 * 1.0e10 / 1.602176634e-19;  // amu (A/fs)^2 -> eV

__device__ __forceinline__ int64_t min_image(int64_t d, int64_t L, int per) {
  if (per) {
    if (2 * d > L) d -= L;
    else if (2 * d < -L) d += L;
  }
  return d;
}

__global__ void bin_kernel(const double *__restrict__ x, int64_t n, Grid g, int4 *__restrict__ q,
                           int32_t *__restrict__ count, int32_t *__restrict__ err) {
  int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n) return;
  int32_t qc[3];
  int64_t cc[3];
  for (int k = 0; k < 3; ++k) {
    long long v = __double2ll_rn(x[3 * o + k] * 1048576.0);
    const long long L = g.Lq[k];
    if (g.per[k]) {
      v %= L;
      if (v < 0) v += L;
    } else if (v < 0 || v >= L) {
      atomicOr(err, ERR_BOUNDS);
      v = v < 0 ? 0 : L - 1;
    }
    qc[k] = (int32_t)v;
    int64_t c = (v * (int64_t)g.nc[k]) / L;
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
__global__ void sort_cells_kernel(const int32_t *__restrict__ start, int64_t ncell,
                                  int32_t *__restrict__ perm) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  int32_t b = start[c], e = start[c + 1];
  for (int32_t i = b + 1; i < e; ++i) {
    int32_t key = perm[i];
    int32_t j = i - 1;
    while (j >= b && perm[j] > key) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = key;
  }
}

// move per-atom data into the new sorted order
__global__ void gather_kernel(int64_t n, const int32_t *__restrict__ perm, const int4 *__restrict__ q,
                              const double *__restrict__ v, const int32_t *__restrict__ type_orig,
                              const int32_t *__restrict__ inv_old, int src_is_orig,
                              const double *__restrict__ T_old, const double *__restrict__ A_old,
                              int32_t *__restrict__ inv_new, int4 *__restrict__ q_s,
                              double *__restrict__ v_s, int8_t *__restrict__ type_s,
                              double *__restrict__ T_new, double *__restrict__ A_new,
                              float *__restrict__ dmir0, double Tref, double invTmax,
                              const double *__restrict__ depth, float *__restrict__ srcw,
                              double inv_lp) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  int32_t o = perm[s];
  q_s[s] = q[o];
  inv_new[o] = (int32_t)s;
  v_s[3 * s + 0] = v[3 * (int64_t)o + 0];
  v_s[3 * s + 1] = v[3 * (int64_t)o + 1];
  v_s[3 * s + 2] = v[3 * (int64_t)o + 2];
  int32_t ty = type_orig ? type_orig[o] : 0;
  type_s[s] = (int8_t)(ty < 0 ? 0 : (ty >= kMaxTypes ? kMaxTypes - 1 : ty));
  int64_t src = src_is_orig ? (int64_t)o : (int64_t)inv_old[o];
  double T = T_old[src];
  T_new[s] = T;
  A_new[s] = A_old[src];
  dmir0[s] = (float)((T - Tref) * invTmax);
  if (srcw) srcw[s] = depth ? (float)exp(-depth[o] * inv_lp) : 0.0f;
}

template <int WMAX>
__global__ void __launch_bounds__(128) neighbor_kernel(int64_t n, Grid g, const int4 *__restrict__ q_s,
                                                       const int32_t *__restrict__ start,
                                                       const int32_t *__restrict__ perm, int32_t W,
                                                       int32_t *__restrict__ nbr, uint8_t *__restrict__ cnt,
                                                       int32_t *__restrict__ maxcnt, int32_t *__restrict__ err) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int4 qi = q_s[s];
  int32_t ci[3];
  ci[0] = qi.w % g.nc[0];
  ci[1] = (qi.w / g.nc[0]) % g.nc[1];
  ci[2] = qi.w / (g.nc[0] * g.nc[1]);
  // distinct neighbour cells per axis (an axis with fewer than 3 cells repeats otherwise)
  int32_t off[3][3];
  int nof[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    nof[k] = 0;
    for (int d = -1; d <= 1; ++d) {
      int32_t c = ci[k] + d;
      if (g.per[k]) {
        if (c < 0) c += g.nc[k];
        if (c >= g.nc[k]) c -= g.nc[k];
      } else if (c < 0 || c >= g.nc[k]) {
        continue;
      }
      bool dup = false;
      for (int m = 0; m < nof[k]; ++m) dup |= (off[k][m] == c);
      if (!dup) off[k][nof[k]++] = c;
    }
  }
  const int64_t rc2 = g.rcq * g.rcq;
  int32_t ct[WMAX];
  int32_t ck[WMAX];
  int32_t m = 0;
  for (int a = 0; a < nof[2]; ++a)
    for (int b = 0; b < nof[1]; ++b)
      for (int d = 0; d < nof[0]; ++d) {
        int32_t cell = off[0][d] + g.nc[0] * (off[1][b] + g.nc[1] * off[2][a]);
        int32_t e = start[cell + 1];
        for (int32_t t = start[cell]; t < e; ++t) {
          if (t == (int32_t)s) continue;
          int4 qj = q_s[t];
          int64_t dx = min_image((int64_t)qj.x - qi.x, g.Lq[0], g.per[0]);
          if (dx > g.rcq || dx < -g.rcq) continue;
          int64_t dy = min_image((int64_t)qj.y - qi.y, g.Lq[1], g.per[1]);
          if (dy > g.rcq || dy < -g.rcq) continue;
          int64_t dz = min_image((int64_t)qj.z - qi.z, g.Lq[2], g.per[2]);
          if (dz > g.rcq || dz < -g.rcq) continue;
          if (dx * dx + dy * dy + dz * dz <= rc2) {
            if (m < W) {
              int32_t key = perm[t];
              // insertion into the row, ascending original id
              int32_t j = m - 1;
              while (j >= 0 && ck[j] > key) {
                ck[j + 1] = ck[j];
                ct[j + 1] = ct[j];
                --j;
              }
              ck[j + 1] = key;
              ct[j + 1] = t;
            }
            ++m;
          }
        }
      }
  if (m > W) atomicOr(err, ERR_NBR_OVERFLOW);
  int32_t mm = m < W ? m : W;
  for (int32_t k = 0; k < mm; ++k) nbr[(int64_t)k * n + s] = ct[k];
  cnt[s] = (uint8_t)mm;
  atomicMax(maxcnt, m);
}

// Sec. 2: T_i^lat = sum_S (1/2) m |v - v_com|^2 / ((3/2) k_B N_j) over S = {i} + neighbours
__global__ void lattice_temp_kernel(int64_t n, const int32_t *__restrict__ nbr,
                                    const uint8_t *__restrict__ cnt, const double *__restrict__ v_s,
                                    const int8_t *__restrict__ type_s, MassTable mt, int dof_mode,
                                    double eps_ke, double *__restrict__ Tl_d, float *__restrict__ Tl_f) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int c = cnt[s];
  double M = 0, px = 0, py = 0, pz = 0;
  for (int k = -1; k < c; ++k) {
    int64_t t = (k < 0) ? s : (int64_t)nbr[(int64_t)k * n + s];
    double m = mt.m[type_s[t]];
    M += m;
    px += m * v_s[3 * t + 0];
    py += m * v_s[3 * t + 1];
    pz += m * v_s[3 * t + 2];
  }
  const double vx = px / M, vy = py / M, vz = pz / M;
  double ke = 0;
  for (int k = -1; k < c; ++k) {
    int64_t t = (k < 0) ? s : (int64_t)nbr[(int64_t)k * n + s];
    double dx = v_s[3 * t + 0] - vx, dy = v_s[3 * t + 1] - vy, dz = v_s[3 * t + 2] - vz;
    ke += 0.5 * mt.m[type_s[t]] * (dx * dx + dy * dy + dz * dz) * kMVV;
  }
  const double dof = (dof_mode == 1) ? (double)c : (double)(c + 1);
  double T = dof > 0 ? ke / (1.5 * kKB * dof) : 0.0;
  const double *vi = v_s + 3 * s;
  double Ks = 0.5 * mt.m[type_s[s]] * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]) * kMVV;
  if (!(Ks >= eps_ke)) T = -1.0;
  Tl_d[s] = T;
  Tl_f[s] = (float)T;
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

// partial sums per block: [0] sum T, [1] max T, [2] sum KE (eV), [3] sum srcw
__global__ void globals_partial(int64_t n, const double *__restrict__ T, const double *__restrict__ v_s,
                                const int8_t *__restrict__ type_s, MassTable mt,
                                const float *__restrict__ srcw, double *__restrict__ part) {
  __shared__ double sh[32];
  double sT = 0, mT = -1e300, sK = 0, sW = 0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    double t = T[s];
    sT += t;
    mT = fmax(mT, t);
    if (v_s) {
      const double *vi = v_s + 3 * s;
      sK += 0.5 * mt.m[type_s[s]] * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]) * kMVV;
    }
    if (srcw) sW += (double)srcw[s];
  }
  double r0 = block_sum(sT, sh);
  double r1 = block_max(mT, sh);
  double r2 = block_sum(sK, sh);
  double r3 = block_sum(sW, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 4 + 0] = r0;
    part[blockIdx.x * 4 + 1] = r1;
    part[blockIdx.x * 4 + 2] = r2;
    part[blockIdx.x * 4 + 3] = r3;
  }
}

__global__ void globals_final(int nb, const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double sh[32];
  double sT = 0, mT = -1e300, sK = 0, sW = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    sT += part[b * 4 + 0];
    mT = fmax(mT, part[b * 4 + 1]);
    sK += part[b * 4 + 2];
    sW += part[b * 4 + 3];
  }
  double r0 = block_sum(sT, sh);
  double r1 = block_max(mT, sh);
  double r2 = block_sum(sK, sh);
  double r3 = block_sum(sW, sh);
  if (threadIdx.x == 0) {
    out[0] = r0;
    out[1] = r1;
    out[2] = r2;
    out[3] = r3;
  }
}

// initial electronic energy per unit volume: int_0^T min(gamma T', cap) dT'
// partials: [0] sum T, [1] max T, [2] sum of the integral [J m^-3], [3] unused
__global__ void seed_partial(int64_t n, const double *__restrict__ T, double gamma, double cap,
                             double *__restrict__ part) {
  __shared__ double sh[32];
  double sT = 0, mT = -1e300, sE = 0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const double t = T[s];
    sT += t;
    mT = fmax(mT, t);
    if (cap > 0.0 && gamma * t > cap) {
      const double Tc = cap / gamma;
      sE += 0.5 * cap * Tc + cap * (t - Tc);
    } else {
      sE += 0.5 * gamma * t * t;
    }
  }
  double r0 = block_sum(sT, sh);
  double r1 = block_max(mT, sh);
  double r2 = block_sum(sE, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 4 + 0] = r0;
    part[blockIdx.x * 4 + 1] = r1;
    part[blockIdx.x * 4 + 2] = r2;
    part[blockIdx.x * 4 + 3] = 0.0;
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
  if (c.n > 0) scatter_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(c.q_orig, c.n, c.cell_start, c.cell_fill, c.perm);
  sort_cells_kernel<<<nblk(c.g.ncell, 256), 256, 0, c.stream>>>(c.cell_start, c.g.ncell, c.perm);
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
        laser ? c.depth_orig : nullptr, c.srcw, laser ? 1.0 / c.p.laser_lp_A : 0.0);
  c.cur_inv = nxt;
  c.tcur = tn;
  double *t = c.A;
  c.A = c.A_tmp;
  c.A_tmp = t;
  c.parity = 0;
  return cudaGetLastError();
}

cudaError_t launch_neighbors(Ctx &c) {
  cudaMemsetAsync(c.maxcnt, 0, sizeof(int32_t), c.stream);
  if (c.n == 0) return cudaGetLastError();
  if (c.W <= 32)
    neighbor_kernel<32><<<nblk(c.n, 128), 128, 0, c.stream>>>(c.n, c.g, c.q_s, c.cell_start, c.perm, c.W,
                                                               c.nbr, c.cnt, c.maxcnt, c.err);
  else
    neighbor_kernel<64><<<nblk(c.n, 128), 128, 0, c.stream>>>(c.n, c.g, c.q_s, c.cell_start, c.perm, c.W,
                                                               c.nbr, c.cnt, c.maxcnt, c.err);
  return cudaGetLastError();
}

cudaError_t launch_lattice_temperature(Ctx &c) {
  if (c.n > 0)
    lattice_temp_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(c.n, c.nbr, c.cnt, c.v_s, c.type_s, c.mt,
                                                              c.p.dof_mode, c.p.eps_ke_eV, c.Tl_d, c.Tl_f);
  return cudaGetLastError();
}

cudaError_t launch_globals(Ctx &c) {
  globals_partial<<<kRedBlocks, kRedThreads, 0, c.stream>>>(c.n, c.T[c.tcur], c.v_s, c.type_s, c.mt,
                                                            (c.p.laser_on && c.have_depth) ? c.srcw : nullptr,
                                                            c.partials);
  globals_final<<<1, kRedThreads, 0, c.stream>>>(kRedBlocks, c.partials, c.scal);
  return cudaGetLastError();
}

cudaError_t launch_ledger(Ctx &c) {
  globals_partial<<<kRedBlocks, kRedThreads, 0, c.stream>>>(c.n, c.T[c.tcur], nullptr, nullptr, c.mt, nullptr,
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
