// kernels_substep.cu -- the per-substep sweep of Eq. HeatTransport.
//
// For every atom i:
//   F_i  = sum_j f(theta_i, theta_j),
//   f(a, b) = b (1 - a) e^{a - b} - a (1 - b) e^{b - a}        (Delta e_ij = -(theta_i - theta_j))
//   T_i += dt [ Tmax K F_i - chi_i (G / C_e)(T_i - T_l,i) + q_i(t) ]
//   A_i += dt chi_i G V_atom (T_i - T_l,i)                    (Eq. RateExchange)
// All atoms read the previous substep's snapshot (Jacobi) through a
// double-buffered mirror.
//
// Single-precision path (flux_prec = 0).
//  * State: delta = (T - Tref) / Tmax held as an unevaluated float pair hi + lo
//    (about 48 significant bits); hi doubles as the mirror the neighbours read.
//    T is rebuilt in FP64 after every substep call (merge) and split again before
//    the next one.  The per-atom exchanged energy A_i is FP64.
//  * Pair term: with a = theta_i, b = theta_j, Delta = b - a and the symmetric
//    P = a + b - 2 a b (so that 2 a (1 - b) = P - Delta and b (1 - a) = a (1 - b) + Delta),
//        f(a, b) = b(1-a) e^{-Delta} - a(1-b) e^{Delta} = Delta cosh(Delta) - P sinh(Delta)
//                = Delta * B,   B = cosh(Delta) - P sinh(Delta)/Delta.
//    B depends on the pair only through Delta^2 and P, which both atoms compute
//    bit for bit alike (fl(a+b) = fl(b+a), and fma(-2a, b, s) = fma(-2b, a, s)),
//    so the two contributions are exactly +-Delta*B: pair fluxes cancel exactly
//    before each atom's own accumulation rounding.  B >= e^{-1} on [0,1]^2, so the
//    FP32 error is relative to the local temperature difference Delta.
//    cosh and sinh(Delta)/Delta come from their Taylor series in Delta^2, with
//    the order set per tile from the largest value spread of its rows (previous
//    substep): spread < 0.02 -> to Delta^2; < 0.12 -> to Delta^4; otherwise to
//    Delta^10 (|Delta| <= 1).  Truncation stays below 3e-8 of B in every tier.
//  * Row tiles: one CTA per row of cells; the rows around it (at most 9) are
//    copied into shared memory and neighbours are 16-bit indices into that tile.
//
// Double-precision path (flux_prec = 1): gathers T itself and evaluates the pair
// term as written in the paper with one exponential, E = e^{theta_lo - theta_hi}:
// f(theta_lo, theta_hi) = theta_hi (1 - theta_lo) E - theta_lo (1 - theta_hi) / E.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

// F += f(theta_i, theta_j) = Delta * B (see above).  ai = theta_i, m2ai = -2 theta_i.
template <int TIER>
__device__ __forceinline__ float pair_acc(float F, float di, float dj, float th, float ai, float m2ai) {
  const float D = dj - di;
  const float x = D * D;
  float S, C;
  if (TIER == 2) {
    S = fmaf(x, 1.6666667e-01f, 1.0f);                              // 1 + D^2/3!
    C = fmaf(x, 0.5f, 1.0f);                                        // 1 + D^2/2!
  } else if (TIER == 1) {
    S = fmaf(x, fmaf(x, 8.3333333e-03f, 1.6666667e-01f), 1.0f);     // ... + D^4/5!
    C = fmaf(x, fmaf(x, 4.1666667e-02f, 0.5f), 1.0f);               // ... + D^4/4!
  } else {
    S = fmaf(x, 2.5052108e-08f, 2.7557319e-06f);                    // 1/11!, 1/9!
    S = fmaf(x, S, 1.9841270e-04f);                                 // 1/7!
    S = fmaf(x, S, 8.3333333e-03f);                                 // 1/5!
    S = fmaf(x, S, 1.6666667e-01f);                                 // 1/3!
    S = fmaf(x, S, 1.0f);
    C = fmaf(x, 2.7557319e-07f, 2.4801587e-05f);                    // 1/10!, 1/8!
    C = fmaf(x, C, 1.3888889e-03f);                                 // 1/6!
    C = fmaf(x, C, 4.1666667e-02f);                                 // 1/4!
    C = fmaf(x, C, 0.5f);
    C = fmaf(x, C, 1.0f);
  }
  const float b = th + dj;
  const float P = fmaf(m2ai, b, ai + b);
  return fmaf(D, fmaf(-P, S, C), F);
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

// (h, l) += x in float-float: TwoSum of h and x, then a fast renormalisation
__device__ __forceinline__ void ff_add(float &h, float &l, float x) {
  const float s = h + x;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (x - bb);
  const float t = l + e;
  const float hn = s + t;
  l = t - (hn - s);
  h = hn;
}

// state update of one atom (single-precision path); returns the new hi
template <bool LASER>
__device__ __forceinline__ float update_atom(int64_t s, float di, float li, float ui, float F,
                                             const StepCoef *__restrict__ cf, float *__restrict__ hout,
                                             float *__restrict__ lo, double *__restrict__ A,
                                             const float *__restrict__ srcw, const float *__restrict__ pulse_f, int k,
                                             int32_t *__restrict__ err) {
  float inc = cf->dtK_f * F;
  const bool chi = (ui == ui);
  float d = 0.0f;
  if (chi) {
    d = fmaf(cf->Tmax_f, di, ui);        // T_i - T_l,i
    inc = fmaf(-cf->dtcGn_f, d, inc);
  }
  float h = di, l = li;
  ff_add(h, l, inc);
  if (LASER) {
    const float c = pulse_f[k], w = srcw[s];
    const float p = c * w;
    const float e = fmaf(c, w, -p);      // p + e == c * w exactly
    ff_add(h, l, p);
    ff_add(h, l, e);
  }
  hout[s] = h;
  lo[s] = l;
  if (chi) A[s] = fma(cf->dtVG, f2d(d), A[s]);
  const float th = cf->th_ref + h;
  if (!(th >= 0.0f && th <= 1.0f)) atomicOr(err, ERR_RANGE);
  return h;
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// Tile descriptor of the row tile around row R of one system.  Neighbour row r
// is placed at tile offset off[r], congruent to its first global index modulo
// 4, so that its interior moves in 16-byte copies.  The system's arguments are
// copied next to it, so every warp reads them from shared memory.
struct TileDesc {
  int32_t start[kRowNbr], len[kRowNbr], off[kRowNbr];
  int32_t self_base, row_s, row_len, tier, row;
  int32_t pad[3];
  RepArgs ra;
};

// computed by one warp: lane r < 9 handles neighbour row r
__device__ __forceinline__ void make_desc(const RepArgs *__restrict__ reps, int2 item, int parity, TileDesc *d) {
  const int lane = threadIdx.x & 31;
  // copy the system's arguments (whole 8-byte words) into the descriptor
  static_assert(sizeof(RepArgs) % 8 == 0, "RepArgs must be a whole number of 8-byte words");
  const uint64_t *src = reinterpret_cast<const uint64_t *>(reps + item.x);
  uint64_t *dst = reinterpret_cast<uint64_t *>(&d->ra);
  for (int w = lane; w < (int)(sizeof(RepArgs) / 8); w += 32) dst[w] = __ldg(src + w);
  __syncwarp();
  const int R = item.y;
  const int32_t ncx = d->ra.ncx;
  const int32_t *row_nbr = d->ra.row_nbr;
  const int32_t *start = d->ra.start;
  const float *rr = d->ra.rrange[parity];
  const int32_t nrows = d->ra.nrows;
  int32_t R2 = -1, a = 0, len = 0;
  float mn = 3.0e38f, mx = -3.0e38f;
  if (lane < kRowNbr) {
    R2 = __ldg(row_nbr + (int64_t)R * kRowNbr + lane);
    if (R2 >= 0) {
      a = __ldg(start + (int64_t)R2 * ncx);
      len = __ldg(start + (int64_t)R2 * ncx + ncx) - a;
      mn = rr[R2];
      mx = rr[nrows + R2];
    }
  }
  // aligned placement, sequential over the 9 rows (same rule as the neighbour build)
  int32_t off = 0, end = 0;
  for (int r = 0; r < kRowNbr; ++r) {
    const int32_t ar = __shfl_sync(0xffffffffu, a, r);
    const int32_t lr = __shfl_sync(0xffffffffu, len, r);
    const int32_t o = end + ((ar - end) & 3);
    if (lane == r) off = o;
    end = o + lr;
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const unsigned selfm = __ballot_sync(0xffffffffu, R2 == R);
  const int sl = __ffs(selfm) - 1;
  if (lane < kRowNbr) {
    d->start[lane] = a;
    d->len[lane] = len;
    d->off[lane] = off;
  }
  if (lane == sl) {
    d->self_base = off;
    d->row_s = a;
    d->row_len = len;
    d->row = R;
    const float spread = mx - mn;
    d->tier = spread < 0.02f ? 2 : (spread < 0.12f ? 1 : 0);
  }
}

// warp w copies neighbour rows w, w + nwarps, ... of hin into buf: unaligned
// head and tail in 4-byte copies, the interior in 16-byte copies
__device__ __forceinline__ void stage_row(const TileDesc *d, const float *hin, float *buf) {
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  for (int w = threadIdx.x >> 5; w < kRowNbr; w += nw) {
    const int32_t a = d->start[w], len = d->len[w];
    float *dst = buf + d->off[w];
    const float *src = hin + a;
    int32_t head = (4 - (a & 3)) & 3;
    if (head > len) head = len;
    if (lane < head) cp_async4(dst + lane, src + lane);
    const int32_t nb = (len - head) >> 2;
    for (int32_t c = lane; c < nb; c += 32) cp_async16(dst + head + 4 * c, src + head + 4 * c);
    const int32_t tail0 = head + 4 * nb;
    if (lane < len - tail0) cp_async4(dst + tail0 + lane, src + tail0 + lane);
  }
}

template <int TIER, bool LASER, int PP>
__device__ __forceinline__ float row_atom(const RepArgs &ra, int parity, int k, const float *tile, int32_t s,
                                          float di, const uint32_t *pv, float ui, float li) {
  const StepCoef *cf = ra.cf;
  const float th = cf->th_ref;
  const float ai = th + di;
  const float m2ai = -2.0f * ai;
  float F = 0.0f;
#pragma unroll
  for (int m = 0; m < PP; ++m)
    if (PP != 16 || m < ra.P) {
      F = pair_acc<TIER>(F, di, tile[pv[m] & 0xffffu], th, ai, m2ai);
      F = pair_acc<TIER>(F, di, tile[pv[m] >> 16], th, ai, m2ai);
    }
  return update_atom<LASER>(s, di, li, ui, F, cf, ra.dmir[parity ^ 1], ra.lo, ra.A, ra.srcw, ra.pulse_f, k,
                            ra.err);
}

// Persistent row-tile kernel over a work list of (system, row) items: each CTA
// walks items blockIdx.x, +gridDim.x, ... and double-buffers the tiles: the
// next item's tile is copied (cp.async) while the current one is computed.
// PP = 9: exactly nine index words per atom (18-neighbour FCC shells) in every
// system; PP = 16: any count up to 32 neighbours, ra.P words.
template <bool LASER, int PP>
__global__ void __launch_bounds__(kTileThreads + 32, kTileMinBlocks)
    substep_tile_kernel(const RepArgs *__restrict__ reps, const int2 *__restrict__ work, int32_t nwork, int32_t tb,
                        int parity, int k) {
  extern __shared__ float tiles[];
  __shared__ TileDesc desc[3];
  __shared__ float wmin[2][kTileThreads / 32], wmax[2][kTileThreads / 32];   // by iteration parity
  int it_item = blockIdx.x;
  if (it_item >= nwork) return;
  const int warp = threadIdx.x >> 5;
  const int aw = kTileThreads / 32;   // warps 0..aw-1 own atoms; warp aw prepares descriptors
  if (warp == 0) make_desc(reps, work[it_item], parity, &desc[0]);
  if (warp == 1 && it_item + (int)gridDim.x < nwork) make_desc(reps, work[it_item + gridDim.x], parity, &desc[1]);
  __syncthreads();
  stage_row(&desc[0], desc[0].ra.dmir[parity], tiles);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  int it = 0;
  // one barrier per item: at the end of an iteration every thread waits for its
  // copies of the next tile, then the barrier makes them (and the descriptor of
  // the item after next) visible and frees the consumed buffer for refilling.
  for (; it_item < nwork; it_item += gridDim.x, ++it) {
    const int dc = it % 3, dn = (it + 1) % 3, dnn = (it + 2) % 3;
    const int buf = it & 1;
    const int nxt = it_item + gridDim.x;
    if (nxt < nwork) stage_row(&desc[dn], desc[dn].ra.dmir[parity], tiles + (buf ^ 1) * tb);
    cp_async_commit();
    if (warp == aw && nxt + (int)gridDim.x < nwork) make_desc(reps, work[nxt + gridDim.x], parity, &desc[dnn]);
    const TileDesc &D = desc[dc];
    const int row_len = D.row_len, row_s = D.row_s, sb = D.self_base;
    const int tier = D.tier;
    const float *tile = tiles + buf * tb;
    float vmin = 3.0e38f, vmax = -3.0e38f;
    for (int q0 = 0; q0 < row_len; q0 += kTileThreads) {
      const int q = q0 + threadIdx.x;
      const bool act = q < row_len && warp < aw;
      const int32_t s = row_s + (act ? q : 0);
      const int32_t n = D.ra.n;
      const uint32_t *pidx = D.ra.pidx;
      uint32_t pv[PP];
#pragma unroll
      for (int m = 0; m < PP; ++m)
        if (PP != 16 || m < D.ra.P) pv[m] = act ? __ldg(pidx + (m * n + s)) : 0u;
      if (act) {
        const float ui = D.ra.uTl[s];
        const float li = D.ra.lo[s];
        const float di = tile[sb + q];
        float h;
        if (tier == 2) h = row_atom<2, LASER, PP>(D.ra, parity, k, tile, s, di, pv, ui, li);
        else if (tier == 1) h = row_atom<1, LASER, PP>(D.ra, parity, k, tile, s, di, pv, ui, li);
        else h = row_atom<0, LASER, PP>(D.ra, parity, k, tile, s, di, pv, ui, li);
        vmin = fminf(vmin, h);
        vmax = fmaxf(vmax, h);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
      vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if ((threadIdx.x & 31) == 0 && warp < aw) {
      wmin[buf][warp] = vmin;
      wmax[buf][warp] = vmax;
    }
    cp_async_wait<0>();
    __syncthreads();
    if (threadIdx.x == 0) {
      float a = wmin[buf][0], b = wmax[buf][0];
      for (int w = 1; w < aw; ++w) {
        a = fminf(a, wmin[buf][w]);
        b = fmaxf(b, wmax[buf][w]);
      }
      float *rr = D.ra.rrange[parity ^ 1];
      rr[D.row] = a;
      rr[D.ra.nrows + D.row] = b;
    }
  }
}

// general single-precision path: one thread per atom, int32 neighbour table,
// neighbour values gathered from global memory (any row length)
template <bool LASER>
__global__ void __launch_bounds__(256) substep_f32_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt,
    const float *__restrict__ hin, float *__restrict__ hout, float *__restrict__ lo, double *__restrict__ A,
    const float *__restrict__ uTl, const float *__restrict__ srcw, const float *__restrict__ pulse_f, int k,
    const StepCoef *__restrict__ cf, int32_t *__restrict__ err) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float th = cf->th_ref;
  const int c = cnt[s];
  const float di = hin[s];
  const float ai = th + di, m2ai = -2.0f * ai;
  float F = 0.0f;
  const int32_t *np = nbr + s;
  int j = 0;
  for (; j + 6 <= c; j += 6) {
    int32_t t[6];
    float dj[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) t[u] = __ldg(np + (int64_t)(j + u) * n);
#pragma unroll
    for (int u = 0; u < 6; ++u) dj[u] = __ldg(hin + t[u]);
#pragma unroll
    for (int u = 0; u < 6; ++u) F = pair_acc<0>(F, di, dj[u], th, ai, m2ai);
  }
  for (; j < c; ++j) F = pair_acc<0>(F, di, __ldg(hin + __ldg(np + (int64_t)j * n)), th, ai, m2ai);
  update_atom<LASER>(s, di, lo[s], uTl[s], F, cf, hout, lo, A, srcw, pulse_f, k, err);
}

// T (FP64) -> hi + lo of delta = (T - Tref) / Tmax
__global__ void split_kernel(int64_t n, const double *__restrict__ T, double Tref, double invTmax,
                             float *__restrict__ hi, float *__restrict__ lo) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double x = (T[s] - Tref) * invTmax;
  const float h = (float)x;
  hi[s] = h;
  lo[s] = (float)(x - (double)h);
}

// hi + lo -> T (FP64)
__global__ void merge_kernel(int64_t n, const float *__restrict__ hi, const float *__restrict__ lo, double Tref,
                             double Tmax, double *__restrict__ T) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  T[s] = Tref + Tmax * ((double)hi[s] + (double)lo[s]);
}

template <bool LASER>
__global__ void __launch_bounds__(256) substep_f64_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt,
    const double *__restrict__ Tin, double *__restrict__ Tout, double *__restrict__ A,
    const double *__restrict__ Tl, const double *__restrict__ srcw, const double *__restrict__ pulse,
    int k, const StepCoef *__restrict__ cf, int32_t *__restrict__ err) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double inv = cf->invTmax;
  const int c = cnt[s];
  const double Ti = Tin[s];
  const double ti = Ti * inv;
  double F = 0.0;
  for (int j = 0; j < c; ++j) {
    const int32_t t = __ldg(nbr + (int64_t)j * n + s);
    const double tj = __ldg(Tin + t) * inv;
    const bool lo = (ti < tj) || (ti == tj && s < t);
    const double a = lo ? ti : tj, b = lo ? tj : ti;
    const double E = exp(a - b);
    const double phi = b * (1.0 - a) * E - a * (1.0 - b) / E;
    F += lo ? phi : -phi;
  }
  double inc = cf->dtTK * F;
  const double tl = Tl[s];
  if (tl >= 0.0) {
    const double d = Ti - tl;
    inc -= cf->dtcG * d;
    A[s] += cf->dtVG * d;
  }
  if (LASER) inc += cf->dt * pulse[k] * srcw[s];
  const double To = Ti + inc;
  Tout[s] = To;
  const double th = To * inv;
  if (!(th >= 0.0 && th <= 1.0)) atomicOr(err, ERR_RANGE);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// the row-tile kernel applies when two tiles fit in shared memory and the table
// holds at most 32 neighbours per atom
bool tile_path(const Ctx &c) {
  return c.p.flux_prec == 0 && c.W <= 32 && c.nwork > 0 && c.staged_max <= c.tile_floats;
}

cudaError_t launch_split(Ctx &c, cudaStream_t st) {
  if (c.n > 0)
    split_kernel<<<nblk(c.n, 256), 256, 0, st>>>(c.n, c.T[c.tcur], c.p.Tref_K, 1.0 / c.p.Tmax_K, c.dmir[c.parity],
                                                 c.dlo);
  return cudaGetLastError();
}

cudaError_t launch_merge(Ctx &c, int parity, cudaStream_t st) {
  if (c.n > 0)
    merge_kernel<<<nblk(c.n, 256), 256, 0, st>>>(c.n, c.dmir[parity], c.dlo, c.p.Tref_K, c.p.Tmax_K, c.T[c.tcur]);
  return cudaGetLastError();
}

// substep k of the current call; parity selects the mirror (FP32) or the T
// buffer (FP64) that holds the previous snapshot.
cudaError_t launch_substep(Ctx &c, int k, int parity, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  const int32_t n = (int32_t)c.n;
  const bool laser = c.p.laser_on && c.have_depth;
  if (c.p.flux_prec == 1) {
    const double *Tin = c.T[parity];
    double *Tout = c.T[parity ^ 1];
    if (laser)
      substep_f64_kernel<true><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, Tin, Tout, c.A, c.Tl_d, c.srcw_d,
                                                             c.pulse, k, c.coef, c.err);
    else
      substep_f64_kernel<false><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, Tin, Tout, c.A, c.Tl_d, c.srcw_d,
                                                              c.pulse, k, c.coef, c.err);
  } else if (tile_path(c)) {
    const int32_t P = (c.n_max + 1) / 2;
    const size_t shm = sizeof(float) * 2 * (size_t)c.tile_floats;
    const unsigned grid = (unsigned)(c.nwork < c.tile_grid ? c.nwork : c.tile_grid);
    if (P == 9) {
      if (laser) substep_tile_kernel<true, 9><<<grid, kTileThreads + 32, shm, st>>>(c.reps, c.work, c.nwork, c.tile_floats, parity, k);
      else substep_tile_kernel<false, 9><<<grid, kTileThreads + 32, shm, st>>>(c.reps, c.work, c.nwork, c.tile_floats, parity, k);
    } else {
      if (laser) substep_tile_kernel<true, 16><<<grid, kTileThreads + 32, shm, st>>>(c.reps, c.work, c.nwork, c.tile_floats, parity, k);
      else substep_tile_kernel<false, 16><<<grid, kTileThreads + 32, shm, st>>>(c.reps, c.work, c.nwork, c.tile_floats, parity, k);
    }
  } else {
    if (laser)
      substep_f32_kernel<true><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, c.dmir[parity], c.dmir[parity ^ 1],
                                                             c.dlo, c.A, c.uTl, c.srcw, c.pulse_f, k, c.coef, c.err);
    else
      substep_f32_kernel<false><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, c.dmir[parity], c.dmir[parity ^ 1],
                                                              c.dlo, c.A, c.uTl, c.srcw, c.pulse_f, k, c.coef,
                                                              c.err);
  }
  return cudaGetLastError();
}

// one substep of the row-tile kernel over an explicit work list (batched systems)
cudaError_t launch_tile_worklist(const RepArgs *reps, const int2 *work, int32_t nwork, int32_t tb, int grid,
                                 int pairs, int parity, int k, cudaStream_t st) {
  const size_t shm = sizeof(float) * 2 * (size_t)tb;
  const unsigned g = (unsigned)(nwork < grid ? nwork : grid);
  if (g == 0) return cudaSuccess;
  if (pairs == 9) substep_tile_kernel<false, 9><<<g, kTileThreads + 32, shm, st>>>(reps, work, nwork, tb, parity, k);
  else substep_tile_kernel<false, 16><<<g, kTileThreads + 32, shm, st>>>(reps, work, nwork, tb, parity, k);
  return cudaGetLastError();
}

// shared memory opt-in and resident CTAs per SM of the tile kernel for two
// buffers of tb floats
cudaError_t tile_setup(int tb, int *blocks_per_sm) {
  const int bytes = (int)(sizeof(float) * 2 * (size_t)tb);
  const void *fns[4] = {(const void *)substep_tile_kernel<true, 9>, (const void *)substep_tile_kernel<false, 9>,
                        (const void *)substep_tile_kernel<true, 16>, (const void *)substep_tile_kernel<false, 16>};
  for (const void *f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  int b9 = 0, b16 = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b9, substep_tile_kernel<false, 9>,
                                                                kTileThreads + 32, (size_t)bytes);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b16, substep_tile_kernel<true, 16>, kTileThreads + 32,
                                                    (size_t)bytes);
  *blocks_per_sm = b9 < b16 ? b9 : b16;
  return e;
}

}  // namespace ehc
