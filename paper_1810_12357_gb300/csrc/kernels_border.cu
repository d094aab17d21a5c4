// kernels_border.cu -- fixed-temperature electron border (a Dirichlet condition
// on T_e, the 300 K border shell of the paper's cascade runs, Sec. 5).
//
// Border atoms (mask 1, sorted order) are electron reservoirs held at their own
// temperature T_b.  The substep kernels take every substep for all atoms (a
// border atom exchanges pair fluxes and coupling energy at its fixed T), then
// store the old value back for border atoms and add the change they would have
// made to the atom's reservoir R (delta units on the single-precision paths,
// kelvin on the FP64 path; times Tmax or 1, times V_atom C_e of the MD step, it
// is the energy the reservoir absorbed).  Here: at each build the reservoirs are
// summed for the ledger of the closing MD step and cleared before the atoms are
// re-sorted; after the new sort the mask is made from the caller-order
// temperatures and border atoms are put to T_b (a difference is charged to R).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr int kBndRedBlocks = 256;

__device__ __forceinline__ double bsum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  return r;
}

// block sums of the reservoirs (grid-stride), clearing them if `clear`
__global__ void __launch_bounds__(256) border_sum_partial(int64_t n, double *__restrict__ R, int clear,
                                                          double *__restrict__ part) {
  __shared__ double sh[8];
  double a = 0.0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    a += R[s];
    if (clear) R[s] = 0.0;
  }
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

// mask of the sorted atoms; border atoms set to T_b, the difference (times
// `scale`: 1 / Tmax for delta units, 1 for kelvin) charged to their reservoir
__global__ void border_mask_kernel(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ tfix,
                                   double *__restrict__ T, double scale, double Tmax, uint8_t *__restrict__ mask,
                                   double *__restrict__ R, int32_t *__restrict__ err) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double t = tfix[perm[s]];
  const bool f = (t == t);
  mask[s] = f ? 1 : 0;
  if (!f) return;
  R[s] += (T[s] - t) * scale;
  T[s] = t;
  if (!(t >= 0.0 && t <= Tmax)) atomicOr(err, ERR_RANGE);
}

}  // namespace

int border_red_blocks() { return kBndRedBlocks; }

cudaError_t border_flush(Ctx &c, double *out, bool clear) {
  border_sum_partial<<<kBndRedBlocks, 256, 0, c.stream>>>(c.n, c.bres, clear ? 1 : 0, c.bnd_part);
  border_sum_final<<<1, 256, 0, c.stream>>>(kBndRedBlocks, c.bnd_part, out);
  return cudaGetLastError();
}

cudaError_t border_apply(Ctx &c) {
  if (c.n > 0) {
    const double scale = c.p.flux_prec == 1 ? 1.0 : 1.0 / c.p.Tmax_K;
    border_mask_kernel<<<(unsigned)((c.n + 255) / 256), 256, 0, c.stream>>>(
        c.n, c.perm, c.tfix_orig, c.T[c.tcur], scale, c.p.Tmax_K, c.bmask, c.bres, c.err);
  }
  return cudaGetLastError();
}

}  // namespace ehc
