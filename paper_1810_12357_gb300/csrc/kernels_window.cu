// kernels_window.cu -- element-wise parts of the Chebyshev window propagator:
// the state as delta = (T - Tref)/Tmax for the stage launches, the accepted
// window's coupling energy, and the a-posteriori residual of a window (the
// stage result goes back to FP64 temperatures in the last stage itself).
//
// A window of n_w substeps of Eq. HeatTransport (pair-flux part) is advanced by
// s stages of the first-order damped Chebyshev recurrence (RKC family):
// Y_1 = Y_0 + mut_1 tau K F(Y_0), Y_j = Y_{j-1} + nu_j (Y_{j-2} - Y_{j-1}) +
// mut_j tau K F(Y_{j-1}).  The stages themselves run in the row-tile kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr int kWinThreads = 256;

__global__ void mirror_kernel(int64_t n, const double *__restrict__ T, double Tref, double invTmax,
                              float *__restrict__ y) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s < n) y[s] = d2f_rn((T[s] - Tref) * invTmax);   // the conversion on the integer pipes
}

// rho_i = |T1 - T0 - tau (R(T0) + R(T1)) / 2| / max(1 K, 1e-3 T0) with
// R = Tmax K F - chi (G/C_e)(T - T_l) (the right-hand side of Eq. HeatTransport).
// Only T1 - T0 is formed in FP64; the rest is single precision, ample for a
// threshold of order one.  Grid-stride loop, block maxima into part.
__global__ void __launch_bounds__(kWinThreads) residual_kernel(int64_t n, const double *__restrict__ T0,
                                                              const double *__restrict__ T1,
                                                              const float *__restrict__ F0,
                                                              const float *__restrict__ F1,
                                                              const float *__restrict__ uTl,
                                                              const StepCoef *__restrict__ cf, float htau,
                                                              float *__restrict__ part) {
  __shared__ float red[kWinThreads / 32];
  const float TK = (float)(cf->dtTK / cf->dt), cG = (float)(cf->dtcG / cf->dt);
  const float Tref = (float)cf->Tref;
  float rho = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float ui = uTl[i];
    const bool chi = ui == ui;
    const double t0 = T0[i], t1 = T1[i];
    const float dT = (float)(t1 - t0);
    const float t0f = (float)t0;
    // T - T_l = (T - Tref) + (Tref - T_l)
    const float c0 = chi ? cG * ((t0f - Tref) + ui) : 0.0f;
    const float c1 = chi ? cG * (((float)t1 - Tref) + ui) : 0.0f;
    const float R = fmaf(TK, F0[i] + F1[i], -(c0 + c1));
    const float r = fabsf(fmaf(-htau, R, dT)) / fmaxf(1.0f, 1e-3f * t0f);
    rho = (r == r) ? fmaxf(rho, r) : 3.0e38f;
  }
  for (int o = 16; o > 0; o >>= 1) rho = fmaxf(rho, __shfl_down_sync(0xffffffffu, rho, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rho;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.0f;
    for (int w = 0; w < kWinThreads / 32; ++w) r = fmaxf(r, red[w]);
    part[blockIdx.x] = r;
  }
}

__global__ void max_kernel(int nb, const float *__restrict__ part, float *__restrict__ out) {
  __shared__ float red[32];
  float r = 0.0f;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) r = fmaxf(r, part[b]);
  for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_down_sync(0xffffffffu, r, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    float x = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x = fmaxf(x, red[w]);
    *out = x;
  }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

constexpr int kResBlocks = 1216;  // 8 x 152 SMs, grid-stride

int cheb_blocks(int64_t n) {
  (void)n;
  return kResBlocks;
}

cudaError_t cheb_mirror(Ctx &c, const double *T, float *y) {
  if (c.n > 0)
    mirror_kernel<<<nblk(c.n, kWinThreads), kWinThreads, 0, c.stream>>>(c.n, T, c.p.Tref_K, 1.0 / c.p.Tmax_K, y);
  return cudaGetLastError();
}

// accepted window: its coupling energy to the ledger A
__global__ void accept_kernel(int64_t n, const double *__restrict__ dTc, double VC, double *__restrict__ A) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double d = dTc[s];
  if ((__double_as_longlong(d) << 1) != 0) A[s] += VC * d;   // d != 0, on the bit pattern
}

cudaError_t cheb_accept(Ctx &c, const double *dTc) {
  if (c.n > 0) accept_kernel<<<nblk(c.n, kWinThreads), kWinThreads, 0, c.stream>>>(c.n, dTc, c.VC, c.A);
  return cudaGetLastError();
}

cudaError_t cheb_residual(Ctx &c, const double *T0, const double *T1, const float *F0, const float *F1, double tau,
                          float *part, float *out) {
  if (c.n == 0) return cudaSuccess;
  residual_kernel<<<kResBlocks, kWinThreads, 0, c.stream>>>(c.n, T0, T1, F0, F1, c.uTl, c.coef, (float)(0.5 * tau),
                                                           part);
  max_kernel<<<1, 256, 0, c.stream>>>(kResBlocks, part, out);
  return cudaGetLastError();
}

}  // namespace ehc
