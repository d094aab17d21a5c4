// kernels_window.cu -- element-wise parts of the Chebyshev window propagator:
// the state as delta = (T - Tref)/Tmax for the stage launches, the stage result
// back to FP64 temperatures, and the a-posteriori residual of a window.
//
// A window of n_w substeps of Eq. HeatTransport (pair-flux part) is advanced by
// s stages of the first-order damped Chebyshev recurrence (RKC family):
// Y_1 = Y_0 + mut_1 tau K F(Y_0), Y_j = Y_{j-1} + nu_j (Y_{j-2} - Y_{j-1}) +
// mut_j tau K F(Y_{j-1}).  The stages themselves run in the row-tile kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr int kWinThreads = 256;

__global__ void mirror_kernel(int64_t n, const double *__restrict__ T, double Tref, double invTmax,
                              float *__restrict__ y) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s < n) y[s] = (float)((T[s] - Tref) * invTmax);
}

__global__ void to_T_kernel(int64_t n, const float *__restrict__ y, double Tref, double Tmax,
                            double *__restrict__ T) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s < n) T[s] = Tref + Tmax * (double)y[s];
}

// rho_i = |T1 - T0 - tau (R(T0) + R(T1)) / 2| / max(1 K, 1e-3 T0) with
// R = Tmax K F - chi (G/C_e)(T - T_l) (the right-hand side of Eq. HeatTransport);
// block maxima into part
__global__ void __launch_bounds__(kWinThreads) residual_kernel(int64_t n, const double *__restrict__ T0,
                                                              const double *__restrict__ T1,
                                                              const float *__restrict__ F0,
                                                              const float *__restrict__ F1,
                                                              const float *__restrict__ uTl,
                                                              const StepCoef *__restrict__ cf, double tau,
                                                              float *__restrict__ part) {
  __shared__ float red[kWinThreads / 32];
  float rho = 0.0f;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const double TK = cf->dtTK / cf->dt, cG = cf->dtcG / cf->dt;
    const float ui = uTl[i];
    const bool chi = ui == ui;
    const double Tl = chi ? cf->Tref - (double)ui : 0.0;
    const double t0 = T0[i], t1 = T1[i];
    const double R0 = TK * (double)F0[i] - (chi ? cG * (t0 - Tl) : 0.0);
    const double R1 = TK * (double)F1[i] - (chi ? cG * (t1 - Tl) : 0.0);
    const double res = fabs(t1 - t0 - 0.5 * tau * (R0 + R1));
    rho = (float)(res / fmax(1.0, 1e-3 * t0));
    if (!(rho == rho)) rho = 3.0e38f;
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

int cheb_blocks(int64_t n) { return (int)nblk(n > 0 ? n : 1, kWinThreads); }

cudaError_t cheb_mirror(Ctx &c, const double *T, float *y) {
  if (c.n > 0)
    mirror_kernel<<<nblk(c.n, kWinThreads), kWinThreads, 0, c.stream>>>(c.n, T, c.p.Tref_K, 1.0 / c.p.Tmax_K, y);
  return cudaGetLastError();
}

cudaError_t cheb_to_T(Ctx &c, const float *y, double *T) {
  if (c.n > 0) to_T_kernel<<<nblk(c.n, kWinThreads), kWinThreads, 0, c.stream>>>(c.n, y, c.p.Tref_K, c.p.Tmax_K, T);
  return cudaGetLastError();
}

cudaError_t cheb_residual(Ctx &c, const double *T0, const double *T1, const float *F0, const float *F1, double tau,
                          float *part, float *out) {
  if (c.n == 0) return cudaSuccess;
  const unsigned nb = nblk(c.n, kWinThreads);
  residual_kernel<<<nb, kWinThreads, 0, c.stream>>>(c.n, T0, T1, F0, F1, c.uTl, c.coef, tau, part);
  max_kernel<<<1, 256, 0, c.stream>>>((int)nb, part, out);
  return cudaGetLastError();
}

}  // namespace ehc
