// kernels_border.cu -- fixed-temperature electron border (a Dirichlet condition
// on T_e, the 300 K border shell of the paper's cascade runs, Sec. 5).
//
// Border atoms (mask 1, sorted order) are electron reservoirs held at their own
// temperature T_b.  The substep kernels take every substep for all atoms (a
// border atom exchanges pair fluxes and coupling energy at its fixed T), then
// store the old value back for border atoms and add the change they would have
// made to the atom's reservoir R (a float pair in delta units on the
// single-precision paths, a double in kelvin on the FP64 path; times Tmax or 1,
// times V_atom C_e of the MD step, it is the energy the reservoir absorbed).  Here: at each build the reservoirs are
// summed for the ledger of the closing MD step and cleared before the atoms are
// re-sorted; after the new sort the mask is made from the caller-order
// temperatures and border atoms are put to T_b (a difference is charged to R).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr int kBndRedBlocks = 2048;   // blocks of 256 threads: enough loads in flight to stream R

__device__ __forceinline__ double bsum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  return r;
}

// block sums of the reservoirs (grid-stride; float pairs if `pairs`, doubles
// otherwise), clearing them if `clear`
__global__ void __launch_bounds__(256) border_sum_partial(int64_t n, double *__restrict__ R, int pairs, int clear,
                                                          double *__restrict__ part) {
  __shared__ double sh[8];
  double a = 0.0;
  float2 *R2 = reinterpret_cast<float2 *>(R);
  // float pairs: each thread sums its pairs as a float pair (single-precision
  // operations) and converts once
  float ah = 0.0f, al = 0.0f;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (pairs) {
      const float2 r = R2[s];
      const float t = ah + r.x, bb = t - ah;
      const float e = (ah - (t - bb)) + (r.x - bb) + (al + r.y);
      ah = t + e;
      al = e - (ah - t);
    } else {
      a += R[s];
    }
    if (clear) R[s] = 0.0;   // both forms: eight zero bytes
  }
  if (pairs) a = (double)ah + (double)al;
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

// mask of the sorted atoms; border atoms set to T_b, the difference charged to
// their (just cleared) reservoir: a float pair of (T - T_b) / Tmax if `pairs`,
// else a double in kelvin
__global__ void border_mask_kernel(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ tfix,
                                   double *__restrict__ T, int pairs, double Tmax, uint8_t *__restrict__ mask,
                                   double *__restrict__ R, int32_t *__restrict__ err) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double t = tfix[perm[s]];
  const bool f = (t == t);
  mask[s] = f ? 1 : 0;
  if (!f) return;
  if (pairs) {
    const double x = (T[s] - t) / Tmax;
    const float hi = (float)x;
    reinterpret_cast<float2 *>(R)[s] = make_float2(hi, (float)(x - (double)hi));
  } else {
    R[s] = T[s] - t;
  }
  T[s] = t;
  if (!(t >= 0.0 && t <= Tmax)) atomicOr(err, ERR_RANGE);
}

}  // namespace

int border_red_blocks() { return kBndRedBlocks; }

cudaError_t border_flush(Ctx &c, double *out, bool clear) {
  border_sum_partial<<<kBndRedBlocks, 256, 0, c.stream>>>(c.n, c.bres, c.p.flux_prec == 0 ? 1 : 0, clear ? 1 : 0,
                                                          c.bnd_part);
  border_sum_final<<<1, 256, 0, c.stream>>>(kBndRedBlocks, c.bnd_part, out);
  return cudaGetLastError();
}

cudaError_t border_apply(Ctx &c) {
  if (c.n > 0) {
    border_mask_kernel<<<(unsigned)((c.n + 255) / 256), 256, 0, c.stream>>>(
        c.n, c.perm, c.tfix_orig, c.T[c.tcur], c.p.flux_prec == 0 ? 1 : 0, c.p.Tmax_K, c.bmask, c.bres, c.err);
  }
  return cudaGetLastError();
}

}  // namespace ehc
