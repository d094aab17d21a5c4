// kernels_halo.cu -- device side of the domain-decomposed design: reading and
// overwriting the electronic temperatures of a list of atoms (caller order)
// between substep calls, for the ghost exchange of the paper's MPI fix
// (ghost-atom temperatures before every substep, Sec. 2.1).
//
// An overwrite keeps the single-precision substep state consistent with T: the
// float pair of delta = (T - Tref)/Tmax (the global form) or of the energy state
// w = u(theta) - u_ref with the mirror (the LOCAL form).  Indices outside
// [0, n) set ERR_INDEX and are skipped (always checked: the list comes from the
// caller).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

__global__ void get_at_kernel(int64_t m, int32_t n, const int32_t *__restrict__ idx, const int32_t *__restrict__ inv,
                              const double *__restrict__ T, double *__restrict__ out, int32_t *__restrict__ err) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int32_t i = idx[k];
  if (i < 0 || i >= n) {
    atomicOr(err, ERR_INDEX);
    out[k] = 0.0;
    return;
  }
  out[k] = T[inv ? inv[i] : i];
}

// mode 0: T only (FP64 path, or a state not yet split); 1: also the float pair of
// delta (hi in mir, lo in lo); 2: the LOCAL form's energy pair (uhi, lo) and mirror
__global__ void set_at_kernel(int64_t m, int32_t n, const int32_t *__restrict__ idx, const int32_t *__restrict__ inv,
                              const double *__restrict__ vals, double *__restrict__ T, float *__restrict__ mir,
                              float *__restrict__ uhi, float *__restrict__ lo, int mode, double Tref,
                              double invTmax, double thc, double u_ref, int32_t *__restrict__ err) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int32_t i = idx[k];
  if (i < 0 || i >= n) {
    atomicOr(err, ERR_INDEX);
    return;
  }
  const int32_t s = inv ? inv[i] : i;
  const double v = vals[k];
  T[s] = v;
  const double x = (v - Tref) * invTmax;
  if (mode == 1) {
    float h, l;
    split_pair(x, h, l);   // as the split of a substep call
    mir[s] = h;
    lo[s] = l;
  } else if (mode == 2) {
    const double w = ue_of(v * invTmax, thc) - u_ref;
    const float h = (float)w;
    uhi[s] = h;
    lo[s] = (float)(w - (double)h);
    mir[s] = (float)x;
  }
}

constexpr int kSumBlocks = 152;   // one block per SM: a fixed grid, deterministic sums
constexpr double kMVVh = 1.66053906660e-27 * 1.0e10 / 1.602176634e-19;   // amu (A/fs)^2 -> eV

__device__ __forceinline__ double hsum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  __syncthreads();
  return r;
}

// block partial sums over the listed atoms: [2b] sum T, [2b + 1] sum of the
// kinetic energy (1/2) m |v|^2 [eV] with the velocities of the last build
__global__ void __launch_bounds__(256) sums_at_partial(int64_t m, int32_t n, const int32_t *__restrict__ idx,
                                                       const int32_t *__restrict__ inv, const double *__restrict__ T,
                                                       const VelQ *__restrict__ v_s, const int8_t *__restrict__ type_s,
                                                       MassTable mt, double *__restrict__ part,
                                                       int32_t *__restrict__ err) {
  __shared__ double sh[8];
  double a = 0.0, b = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = idx[k];
    if (i < 0 || i >= n) {
      atomicOr(err, ERR_INDEX);
      continue;
    }
    const int32_t s = inv[i];
    a += T[s];
    b += 0.5 * mt.m[type_s[s]] * v_s[s].w * kMVVh;
  }
  const double ra = hsum(a, sh);
  const double rb = hsum(b, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ra;
    part[2 * blockIdx.x + 1] = rb;
  }
}

__global__ void __launch_bounds__(256) sums_at_final(const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double sh[8];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < kSumBlocks; k += blockDim.x) {
    a += part[2 * k];
    b += part[2 * k + 1];
  }
  const double ra = hsum(a, sh);
  const double rb = hsum(b, sh);
  if (threadIdx.x == 0) {
    out[0] = ra;
    out[1] = rb;
  }
}

inline unsigned hblk(int64_t m) { return (unsigned)((m + 255) / 256); }

}  // namespace

cudaError_t launch_get_at(Ctx &c, const int32_t *idx, int64_t m, double *out) {
  if (m > 0)
    get_at_kernel<<<hblk(m), 256, 0, c.stream>>>(m, (int32_t)c.n, idx, c.te_orig_order ? nullptr : c.inv_perm[c.cur_inv],
                                                  c.T[c.tcur], out, c.err);
  return cudaGetLastError();
}

cudaError_t launch_set_at(Ctx &c, const int32_t *idx, int64_t m, const double *vals) {
  if (m <= 0) return cudaSuccess;
  int mode = 0;
  if (c.p.flux_prec == 0 && c.ff_valid && !c.te_orig_order) mode = c.local ? 2 : 1;
  const StepCoef &cf = *c.coef_host;
  set_at_kernel<<<hblk(m), 256, 0, c.stream>>>(m, (int32_t)c.n, idx, c.te_orig_order ? nullptr : c.inv_perm[c.cur_inv],
                                               vals, c.T[c.tcur], c.dmir[c.parity], c.uhi, c.dlo, mode, c.p.Tref_K,
                                               1.0 / c.p.Tmax_K, cf.thc, cf.u_ref, c.err);
  return cudaGetLastError();
}

cudaError_t launch_sums_at(Ctx &c, const int32_t *idx, int64_t m, double *part, double *out) {
  sums_at_partial<<<kSumBlocks, 256, 0, c.stream>>>(m, (int32_t)c.n, idx, c.inv_perm[c.cur_inv], c.T[c.tcur], c.v_s,
                                                    c.type_s, c.mt, part, c.err);
  sums_at_final<<<1, 256, 0, c.stream>>>(part, out);
  return cudaGetLastError();
}

}  // namespace ehc
