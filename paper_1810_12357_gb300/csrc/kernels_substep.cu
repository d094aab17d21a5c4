// kernels_substep.cu -- the per-substep sweep of Eq. HeatTransport.
//
// For every atom i (one thread per atom, atoms in cell-sorted order):
//   F_i  = sum_j f(theta_i, theta_j),
//   f(a, b) = b (1 - a) e^{a - b} - a (1 - b) e^{b - a}        (Delta e_ij = -(theta_i - theta_j))
//   T_i += dt [ Tmax K F_i - chi_i (G / C_e)(T_i - T_l,i) + q_i(t) ]
//   A_i += dt chi_i G V_atom (T_i - T_l,i)                    (Eq. RateExchange)
// All atoms read the previous substep's snapshot (Jacobi), through a
// double-buffered mirror.
//
// Canonical pair evaluation: the pair {i, j} is always evaluated as
// f(theta_lo, theta_hi) with lo the smaller sorted index; the atom that is
// 'hi' adds the negated value.  Both atoms run the same instructions on the
// same operands, so the two contributions cancel bit for bit and the flux part
// of sum_i T_i is conserved up to the rounding of each atom's own sum.
//
// FP32 path.  The mirror holds delta = (T - Tref) / Tmax in FP32 and with
// Delta = delta_hi - delta_lo, a = Tref/Tmax + delta_lo, b = Tref/Tmax + delta_hi:
//   f(a, b) = Delta e^{-Delta} - 2 a (1 - b) sinh(Delta)
// (since b(1-a) = a(1-b) + Delta).  The leading term is Delta times a factor of
// order one, so the FP32 error is relative to the local temperature difference
// rather than to T itself.  sinh and cosh come from their Taylor series to
// order 11 and 10 (|Delta| <= 1, truncation below 3e-9 relative); e^{-Delta} =
// cosh - sinh.  No special-function unit is used.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

__device__ __forceinline__ float pair_flux_f32(float dlo, float dhi, float th_ref) {
  const float D = dhi - dlo;
  const float D2 = D * D;
  float S = fmaf(D2, 2.5052108e-08f, 2.7557319e-06f);   // 1/11!, 1/9!
  S = fmaf(D2, S, 1.9841270e-04f);                      // 1/7!
  S = fmaf(D2, S, 8.3333333e-03f);                      // 1/5!
  S = fmaf(D2, S, 1.6666667e-01f);                      // 1/3!
  S = fmaf(D2, S, 1.0f);
  float C = fmaf(D2, 2.7557319e-07f, 2.4801587e-05f);   // 1/10!, 1/8!
  C = fmaf(D2, C, 1.3888889e-03f);                      // 1/6!
  C = fmaf(D2, C, 4.1666667e-02f);                      // 1/4!
  C = fmaf(D2, C, 0.5f);
  C = fmaf(D2, C, 1.0f);
  const float sh = D * S;
  const float em = C - sh;
  const float a = th_ref + dlo;
  const float b = th_ref + dhi;
  const float w = 2.0f * a * (1.0f - b);
  return fmaf(D, em, -(w * sh));
}

constexpr int kBatch = 6;

template <bool LASER>
__global__ void __launch_bounds__(256) substep_f32_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt,
    const float *__restrict__ din, float *__restrict__ dout, double *__restrict__ T,
    double *__restrict__ A, const float *__restrict__ Tl, const float *__restrict__ srcw,
    const double *__restrict__ pulse, int k, const StepCoef *__restrict__ cf,
    int32_t *__restrict__ err) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float th_ref = cf->th_ref;
  const int c = cnt[s];
  const float di = din[s];
  float F = 0.0f;
  const int32_t *np = nbr + s;
  int j = 0;
  for (; j + kBatch <= c; j += kBatch) {
    int32_t t[kBatch];
    float dj[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) t[u] = __ldg(np + (int64_t)(j + u) * n);
#pragma unroll
    for (int u = 0; u < kBatch; ++u) dj[u] = __ldg(din + t[u]);
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const bool lo = s < t[u];
      const float phi = pair_flux_f32(lo ? di : dj[u], lo ? dj[u] : di, th_ref);
      F += lo ? phi : -phi;
    }
  }
  for (; j < c; ++j) {
    const int32_t t = __ldg(np + (int64_t)j * n);
    const float dj = __ldg(din + t);
    const bool lo = s < t;
    const float phi = pair_flux_f32(lo ? di : dj, lo ? dj : di, th_ref);
    F += lo ? phi : -phi;
  }
  double Ti = T[s];
  double inc = cf->dtTK * (double)F;
  const float tl = Tl[s];
  if (tl >= 0.0f) {
    const double d = Ti - (double)tl;
    inc = fma(-cf->dtcG, d, inc);
    A[s] = fma(cf->dtVG, d, A[s]);
  }
  if (LASER) inc = fma(cf->dt * pulse[k], (double)srcw[s], inc);
  Ti += inc;
  T[s] = Ti;
  const float dn = (float)((Ti - cf->Tref) * cf->invTmax);
  dout[s] = dn;
  const float th = th_ref + dn;
  if (!(th >= 0.0f && th <= 1.0f)) atomicOr(err, ERR_RANGE);
}

// FP64 path: gathers T itself, evaluates the pair term as written in the
// paper with one exponential: E = e^{theta_lo - theta_hi},
// f(theta_lo, theta_hi) = theta_hi (1 - theta_lo) E - theta_lo (1 - theta_hi) / E.
template <bool LASER>
__global__ void __launch_bounds__(256) substep_f64_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt,
    const double *__restrict__ Tin, double *__restrict__ Tout, double *__restrict__ A,
    const double *__restrict__ Tl, const float *__restrict__ srcw, const double *__restrict__ pulse,
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
    const bool lo = s < t;
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
  if (LASER) inc += cf->dt * pulse[k] * (double)srcw[s];
  const double To = Ti + inc;
  Tout[s] = To;
  const double th = To * inv;
  if (!(th >= 0.0 && th <= 1.0)) atomicOr(err, ERR_RANGE);
}

}  // namespace

// substep k of the current call; parity selects the mirror (FP32) or the T
// buffer (FP64) that holds the previous snapshot.
cudaError_t launch_substep(Ctx &c, int k, int parity, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  const int32_t n = (int32_t)c.n;
  const unsigned nb = (unsigned)((c.n + 255) / 256);
  const bool laser = c.p.laser_on && c.have_depth;
  if (c.p.flux_prec == 1) {
    const double *Tin = c.T[parity];
    double *Tout = c.T[parity ^ 1];
    if (laser)
      substep_f64_kernel<true><<<nb, 256, 0, st>>>(n, c.nbr, c.cnt, Tin, Tout, c.A, c.Tl_d, c.srcw, c.pulse, k,
                                                   c.coef, c.err);
    else
      substep_f64_kernel<false><<<nb, 256, 0, st>>>(n, c.nbr, c.cnt, Tin, Tout, c.A, c.Tl_d, c.srcw, c.pulse, k,
                                                    c.coef, c.err);
  } else {
    if (laser)
      substep_f32_kernel<true><<<nb, 256, 0, st>>>(n, c.nbr, c.cnt, c.dmir[parity], c.dmir[parity ^ 1],
                                                   c.T[c.tcur], c.A, c.Tl_f, c.srcw, c.pulse, k, c.coef, c.err);
    else
      substep_f32_kernel<false><<<nb, 256, 0, st>>>(n, c.nbr, c.cnt, c.dmir[parity], c.dmir[parity ^ 1],
                                                    c.T[c.tcur], c.A, c.Tl_f, c.srcw, c.pulse, k, c.coef, c.err);
  }
  return cudaGetLastError();
}

}  // namespace ehc
