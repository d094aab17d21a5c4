// kernels_border.cu -- fixed-temperature electron border (a Dirichlet condition
// on T_e, the 300 K border shell of the paper's cascade runs, Sec. 5).
//
// Border atoms are electron reservoirs held at their own temperature T_b.  Each
// substep is taken for every atom as usual (a border atom exchanges pair fluxes
// and coupling energy with its T held at T_b); afterwards the atoms of the
// border list are put back to T_b, and the change they would have made,
// T_new - T_b, is added to a per-atom reservoir R (kelvin; times V_atom C_e of
// the MD step it is the energy the reservoir absorbed).  The list is rebuilt in
// sorted order at every neighbour build (counts per block, one-block scan,
// ballot-ranked scatter), after the previous list's reservoirs have been summed.
// The row value ranges that choose the next substep's Taylor tier are widened
// to include the reset values (the substep kernel recorded the values before
// the reset).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr int kBndBlock = 1024;
constexpr int kBndFixThreads = 256;
constexpr int kBndFixMaxBlocks = 8192;   // one entry per thread up to 2M entries, then grid-stride
constexpr int kBndRedBlocks = 256;

__device__ __forceinline__ bool fixed_value(double t) { return t == t; }

// number of border atoms among sorted atoms [b 1024, (b + 1) 1024)
__global__ void __launch_bounds__(kBndBlock) border_count_kernel(int64_t n, const int32_t *__restrict__ perm,
                                                                 const double *__restrict__ tfix,
                                                                 int32_t *__restrict__ cnt) {
  __shared__ int32_t wc[kBndBlock / 32];
  const int64_t s = blockIdx.x * (int64_t)kBndBlock + threadIdx.x;
  const bool f = s < n && fixed_value(tfix[perm[s]]);
  const unsigned b = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < kBndBlock / 32; ++w) t += wc[w];
    cnt[blockIdx.x] = t;
  }
}

// exclusive offsets of the nb block counts, and their total (one block)
__global__ void __launch_bounds__(1024) border_offsets_kernel(int nb, const int32_t *__restrict__ cnt,
                                                              int32_t *__restrict__ off, int32_t *__restrict__ total) {
  __shared__ int32_t ws[32];
  const int t = threadIdx.x;
  const int per = (nb + 1023) / 1024;
  const int b0 = t * per, b1 = min(nb, b0 + per);
  int32_t sum = 0;
  for (int b = b0; b < b1; ++b) sum += cnt[b];
  // inclusive scan of the chunk sums over the block
  int32_t x = sum;
  const int lane = t & 31, w = t >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t v = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    ws[lane] = v;
  }
  __syncthreads();
  const int32_t incl = x + (w > 0 ? ws[w - 1] : 0);
  int32_t run = incl - sum;
  for (int b = b0; b < b1; ++b) {
    off[b] = run;
    run += cnt[b];
  }
  if (t == 1023) *total = incl;
}

// the list in sorted order: entry k holds the sorted index, T_b as a float pair
// of (T_b - Tref)/Tmax (the split of the single-precision state) and in FP64,
// and a zeroed reservoir
__global__ void __launch_bounds__(kBndBlock) border_scatter_kernel(
    int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ tfix, const int32_t *__restrict__ off,
    const int4 *__restrict__ q_s, int32_t ncx, double Tref, double invTmax, double Tmax, int32_t *__restrict__ bs,
    int32_t *__restrict__ brow, float *__restrict__ bh, float *__restrict__ bl, double *__restrict__ bT,
    double *__restrict__ R, int32_t *__restrict__ err) {
  __shared__ int32_t wo[kBndBlock / 32];
  const int64_t s = blockIdx.x * (int64_t)kBndBlock + threadIdx.x;
  const double t = s < n ? tfix[perm[s]] : 0.0;
  const bool f = s < n && fixed_value(t);
  const unsigned b = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wo[w] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int k = 0; k < kBndBlock / 32; ++k) {
      const int32_t c = wo[k];
      wo[k] = run;
      run += c;
    }
  }
  __syncthreads();
  if (!f) return;
  const int32_t k = off[blockIdx.x] + wo[w] + __popc(b & ((1u << lane) - 1u));
  bs[k] = (int32_t)s;
  brow[k] = q_s[s].w / ncx;   // the atom's cell row (the row tiles' unit)
  const double x = (t - Tref) * invTmax;
  const float h = (float)x;
  bh[k] = h;
  bl[k] = (float)(x - (double)h);
  bT[k] = t;
  R[k] = 0.0;
  if (!(t >= 0.0 && t <= Tmax)) atomicOr(err, ERR_RANGE);
}

// *a = min(*a, v) and *a = max(*a, v) on floats by compare-and-swap; each round
// lets one writer through, so a row's writers (at most the atoms of the row)
// finish within that many rounds
constexpr int kCasRounds = 4096;
__device__ __forceinline__ void atomic_fmin(float *a, float v) {
  int *ai = reinterpret_cast<int *>(a);
  int old = *ai;
  for (int it = 0; it < kCasRounds && __int_as_float(old) > v; ++it) {
    const int prev = atomicCAS(ai, old, __float_as_int(v));
    if (prev == old) break;
    old = prev;
  }
}
__device__ __forceinline__ void atomic_fmax(float *a, float v) {
  int *ai = reinterpret_cast<int *>(a);
  int old = *ai;
  for (int it = 0; it < kCasRounds && __int_as_float(old) < v; ++it) {
    const int prev = atomicCAS(ai, old, __float_as_int(v));
    if (prev == old) break;
    old = prev;
  }
}

__global__ void __launch_bounds__(kBndFixThreads) border_fix_f32_kernel(
    const int32_t *__restrict__ bn, const int32_t *__restrict__ bs, const int32_t *__restrict__ brow,
    const float *__restrict__ bh, const float *__restrict__ bl, float *__restrict__ hout, float *__restrict__ lo,
    double *__restrict__ R, double Tmax, int32_t nrows, float *__restrict__ rr) {
  const int32_t m = *bn;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const int32_t s = bs[k];
    const float hb = bh[k], lb = bl[k];
    const double d = ((double)hout[s] - (double)hb) + ((double)lo[s] - (double)lb);
    R[k] += Tmax * d;
    hout[s] = hb;
    lo[s] = lb;
    if (rr) {
      // usually inside the row's range already: then no atomic is issued
      const int32_t row = brow[k];
      atomic_fmin(rr + row, hb);
      atomic_fmax(rr + nrows + row, hb);
    }
  }
}

__global__ void __launch_bounds__(kBndFixThreads) border_fix_f64_kernel(
    const int32_t *__restrict__ bn, const int32_t *__restrict__ bs, const double *__restrict__ bT,
    double *__restrict__ Tout, double *__restrict__ R) {
  const int32_t m = *bn;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const int32_t s = bs[k];
    R[k] += Tout[s] - bT[k];
    Tout[s] = bT[k];
  }
}

__device__ __forceinline__ double bsum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  return r;
}

// sum of the reservoirs of the current list: block sums, then one block in order
__global__ void __launch_bounds__(256) border_sum_partial(const int32_t *__restrict__ bn,
                                                          const double *__restrict__ R, double *__restrict__ part) {
  __shared__ double sh[8];
  const int32_t m = *bn;
  double a = 0.0;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) a += R[k];
  const double r = bsum(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void __launch_bounds__(256) border_sum_final(int nb, const double *__restrict__ part,
                                                        double *__restrict__ out) {
  __shared__ double sh[8];
  double a = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) a += part[k];
  const double r = bsum(a, sh);
  if (threadIdx.x == 0) *out = r;
}

}  // namespace

int border_blocks(int64_t n) { return (int)((n + kBndBlock - 1) / kBndBlock); }
int border_red_blocks() { return kBndRedBlocks; }

cudaError_t border_sum(Ctx &c, double *out) {
  border_sum_partial<<<kBndRedBlocks, 256, 0, c.stream>>>(c.bnd_n, c.bnd_R, c.bnd_part);
  border_sum_final<<<1, 256, 0, c.stream>>>(kBndRedBlocks, c.bnd_part, out);
  return cudaGetLastError();
}

cudaError_t border_build(Ctx &c) {
  if (c.n == 0) return cudaMemsetAsync(c.bnd_n, 0, sizeof(int32_t), c.stream);
  const int nb = border_blocks(c.n);
  border_count_kernel<<<nb, kBndBlock, 0, c.stream>>>(c.n, c.perm, c.tfix_orig, c.bnd_cnt);
  border_offsets_kernel<<<1, 1024, 0, c.stream>>>(nb, c.bnd_cnt, c.bnd_off, c.bnd_n);
  border_scatter_kernel<<<nb, kBndBlock, 0, c.stream>>>(c.n, c.perm, c.tfix_orig, c.bnd_off, c.q_s, c.g.nc[0],
                                                        c.p.Tref_K, 1.0 / c.p.Tmax_K, c.p.Tmax_K, c.bnd_s,
                                                        c.bnd_row, c.bnd_h, c.bnd_l, c.bnd_T, c.bnd_R, c.err);
  return cudaGetLastError();
}

cudaError_t border_fix(Ctx &c, int parity, bool tile, cudaStream_t st) {
  // the grid covers the list's capacity (the count is known on the device only,
  // and captured graphs replay the launch as it was recorded)
  int64_t b = (c.n + kBndFixThreads - 1) / kBndFixThreads;
  const unsigned grid = (unsigned)(b < 1 ? 1 : (b > kBndFixMaxBlocks ? kBndFixMaxBlocks : b));
  if (c.p.flux_prec == 1) {
    border_fix_f64_kernel<<<grid, kBndFixThreads, 0, st>>>(c.bnd_n, c.bnd_s, c.bnd_T, c.T[parity ^ 1], c.bnd_R);
  } else {
    border_fix_f32_kernel<<<grid, kBndFixThreads, 0, st>>>(c.bnd_n, c.bnd_s, c.bnd_row, c.bnd_h, c.bnd_l,
                                                           c.dmir[parity ^ 1], c.dlo, c.bnd_R, c.p.Tmax_K,
                                                           (int32_t)c.nrows, tile ? c.rrange[parity ^ 1] : nullptr);
  }
  return cudaGetLastError();
}

}  // namespace ehc
