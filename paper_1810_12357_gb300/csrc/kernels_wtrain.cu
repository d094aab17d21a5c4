// kernels_wtrain.cu -- training of the Chebyshev window's stage coefficients:
// every stage of a window on the neighbour list (kept for the backward sweep),
// the window loss, the adjoint sweep, the gradient reductions and Adam.
//
// Values are delta = (T - Tref)/Tmax, theta = Tref/Tmax + delta.  On the window's
// change z_j = Y_j - Y_0 (z_0 = 0), with a_j = mut_j tau K and g_j = gam_j tau K:
//   z_1 = a_1 F(Y_0),
//   z_j = z_{j-1} + nu_j (z_{j-2} - z_{j-1}) - kap_j z_{j-1} + a_j F(Y_{j-1}) + g_j F(Y_0),
// F_i = sum_j f(theta_i, theta_j) the pair flux of Eq. HeatTransport, evaluated as
// f(a, b) = D cosh D - P sinh D with D = b - a, P = a + b - 2ab.
// Loss of a window against the plain method's end state T1 (p = 2, 4 or 8; the
// higher powers weigh the atoms with the largest errors):
//   L = mean_i ((T0_i + Tmax z_s,i - T1_i) / T0_i)^p.
// Adjoint lam_j = dL/dz_j, from j = s down:
//   lam_{j-1} += (1 - nu_j - kap_j) lam_j + a_j J(Y_{j-1})^T lam_j,  lam_{j-2} += nu_j lam_j,
//   dL/dnu_j = <lam_j, z_{j-2} - z_{j-1}>, dL/dkap_j = -<lam_j, z_{j-1}>,
//   dL/dmut_j = tau K <lam_j, F(Y_{j-1})>, dL/dgam_j = tau K <lam_j, F(Y_0)>.
// The neighbour list is symmetric and f is odd, so the transposed Jacobian is a
// gather over atom m's own row:
//   (J^T lam)_m = sum_{j in row m} (lam_m - lam_j) d_a f(theta_m, theta_j),
//   d_a f(a, b) = -((1 - P) cosh D + (1 - S) sinh D),  S = a + b.
// Single precision throughout except the FP64 temperatures and the FP64
// reductions of the loss and the gradient.  One thread per atom (training runs
// on windows of a few hundred thousand atoms; the product path is the row-tile
// kernel).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr int kWtThreads = 256;
constexpr int kWtDotBlocks = 608;   // 4 x 152 SMs, grid-stride

inline unsigned wblk(int64_t n) { return (unsigned)((n + kWtThreads - 1) / kWtThreads); }

__device__ __forceinline__ float pair_f(float a, float b) {
  const float D = b - a;
  const float P = fmaf(-2.0f * a, b, a + b);
  return fmaf(D, coshf(D), -P * sinhf(D));
}

__device__ __forceinline__ float pair_da(float a, float b) {
  const float D = b - a;
  const float S = a + b;
  const float P = fmaf(-2.0f * a, b, S);
  return -fmaf(1.0f - P, coshf(D), (1.0f - S) * sinhf(D));
}

// one stage: F(Y_{j-1}) into Fout and z_j into zout (zm1 == nullptr: stage 1)
__global__ void __launch_bounds__(kWtThreads) wt_stage_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt, float th,
    const float *__restrict__ y0, const float *__restrict__ zm1, const float *__restrict__ zm2,
    const float *__restrict__ F0, float nu, float kap, float a, float g, float *__restrict__ Fout,
    float *__restrict__ zout) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float z1 = zm1 ? zm1[i] : 0.0f;
  const float ai = th + (y0[i] + z1);
  float F = 0.0f;
  const int ci = cnt[i];
  for (int e = 0; e < ci; ++e) {
    const int32_t j = __ldg(nbr + (int64_t)e * n + i);
    const float yj = __ldg(y0 + j) + (zm1 ? __ldg(zm1 + j) : 0.0f);
    F += pair_f(ai, th + yj);
  }
  Fout[i] = F;
  if (!zm1) {
    zout[i] = a * F;
    return;
  }
  const float z2 = zm2 ? zm2[i] : 0.0f;
  const float f0 = F0 ? F0[i] : 0.0f;
  const float inc = fmaf(g, f0, fmaf(-kap, z1, a * F));
  zout[i] = z1 + fmaf(nu, z2 - z1, inc);
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) r += red[w];
  __syncthreads();
  return r;
}

// r_i = (T0 + Tmax z_s - T1) / T0, loss mean r^p (p = 2, 4, 8):
// lam_s = dL/dz_s = p r^(p-1) Tmax / (n T0), block sums of r^p
__global__ void __launch_bounds__(kWtThreads) wt_loss_kernel(int32_t n, const float *__restrict__ zs,
                                                            const double *__restrict__ T0,
                                                            const double *__restrict__ T1, double Tmax, int pw,
                                                            float *__restrict__ lam, double *__restrict__ part) {
  __shared__ double red[kWtThreads / 32];
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double rp = 0.0;
  if (i < n) {
    const double t0 = T0[i];
    const double r = (fma(Tmax, (double)zs[i], t0) - T1[i]) / t0;
    double rq = r;   // r^(p-1)
    for (int k = 2; k < pw; ++k) rq *= r;
    rp = rq * r;
    lam[i] = (float)(pw * rq * Tmax / ((double)n * t0));
  }
  const double b = block_sum<kWtThreads>(rp, red);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// stage j of the backward sweep: lam1 = lam_{j-1} += c1 lam_j + a (J(Y_{j-1})^T lam_j),
// lam2 = lam_{j-2} += nu lam_j (lam2 == nullptr when j - 2 = 0); for rollouts
// also mu += a J(Y_{j-1})^T lam_j and gs += g lam_j (the window-start adjoint's
// parts; null when not wanted)
__global__ void __launch_bounds__(kWtThreads) wt_adjoint_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt, float th,
    const float *__restrict__ y0, const float *__restrict__ zm1, const float *__restrict__ lam, float c1, float a,
    float nu, float *__restrict__ lam1, float *__restrict__ lam2, float g = 0.0f, float *__restrict__ mu = nullptr,
    float *__restrict__ gs = nullptr) {
  const int32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const float am = th + (y0[m] + zm1[m]);
  const float lm = lam[m];
  float acc = 0.0f;
  const int cm = cnt[m];
  for (int e = 0; e < cm; ++e) {
    const int32_t j = __ldg(nbr + (int64_t)e * n + m);
    const float bj = th + (__ldg(y0 + j) + __ldg(zm1 + j));
    acc = fmaf(lm - __ldg(lam + j), pair_da(am, bj), acc);
  }
  lam1[m] += fmaf(a, acc, c1 * lm);
  if (lam2) lam2[m] += nu * lm;
  if (mu) mu[m] += a * acc;
  if (gs) gs[m] += g * lm;
}

// per stage j = blockIdx.y + 1 the four inner products of the gradient, block
// sums into part[(4 j + q) * gridDim.x + blockIdx.x]
__global__ void __launch_bounds__(kWtThreads) wt_dots_kernel(int32_t n, WtTab t, double *__restrict__ part,
                                                            int accumulate = 0) {
  __shared__ double red[kWtThreads / 32];
  const int j = blockIdx.y + 1;
  const float *lam = t.lam[j];
  const float *Fj = t.F[j];
  const float *F0 = t.F[1];
  const float *z1 = j >= 2 ? t.z[j - 1] : nullptr;
  const float *z2 = j >= 3 ? t.z[j - 2] : nullptr;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double l = lam[i];
    const double a1 = z1 ? z1[i] : 0.0, a2 = z2 ? z2[i] : 0.0;
    s0 += l * (a2 - a1);
    s1 += l * Fj[i];
    s2 -= l * a1;
    s3 += l * F0[i];
  }
  const double v0 = block_sum<kWtThreads>(s0, red);
  const double v1 = block_sum<kWtThreads>(s1, red);
  const double v2 = block_sum<kWtThreads>(s2, red);
  const double v3 = block_sum<kWtThreads>(s3, red);
  if (threadIdx.x == 0) {
    const size_t base = (size_t)4 * j * gridDim.x + blockIdx.x;
    if (accumulate) {
      part[base] += v0;
      part[base + gridDim.x] += v1;
      part[base + 2 * gridDim.x] += v2;
      part[base + 3 * gridDim.x] += v3;
    } else {
      part[base] = v0;
      part[base + gridDim.x] = v1;
      part[base + 2 * gridDim.x] = v2;
      part[base + 3 * gridDim.x] = v3;
    }
  }
}

// gradient entry (q, j) per block (q: nu, mut, kap, gam), the last block the loss:
// gc = dL/dc (the tau K factor for mut and gam; stage 1 only has mut), and, for
// Adam on the relative changes d (c = c0 (1 + d)), gd = gc c0
__global__ void wt_final_kernel(int s, int nbd, const double *__restrict__ part, int nbl,
                                const double *__restrict__ lpart, double tauK, double inv_n,
                                const float *__restrict__ c0, float *__restrict__ gc, float *__restrict__ gd,
                                float *__restrict__ loss) {
  __shared__ double red[4];
  const int b = blockIdx.x;
  const int np = 4 * (s + 1);
  double acc = 0.0;
  if (b == np) {
    for (int k = threadIdx.x; k < nbl; k += blockDim.x) acc += lpart[k];
  } else {
    const int q = b / (s + 1), j = b % (s + 1);
    if (j >= 1)
      for (int k = threadIdx.x; k < nbd; k += blockDim.x) acc += part[((size_t)4 * j + q) * nbd + k];
  }
  const double v = block_sum<128>(acc, red);
  if (threadIdx.x != 0) return;
  if (b == np) {
    *loss = (float)(v * inv_n);
    return;
  }
  const int q = b / (s + 1), j = b % (s + 1);
  double g = (q == 1 || q == 3) ? v * tauK : v;
  if (j == 0 || (j == 1 && q != 1)) g = 0.0;
  gc[b] = (float)g;
  gd[b] = c0[b] != 0.0f ? (float)(g * (double)c0[b]) : 0.0f;
}

__global__ void wt_adam_kernel(int np, float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                               const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1,
                               float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const float gk = g[k];
  const float mk = fmaf(b1, m[k], (1.0f - b1) * gk);
  const float vk = fmaf(b2, v[k], (1.0f - b2) * gk * gk);
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// power iteration on J^T: a start vector without a uniform part (hash of the atom
// index), sums of squares, and the normalisation v = u / |u|
__global__ void wt_seed_kernel(int32_t n, float *__restrict__ v) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t h = (uint32_t)i * 0x9E3779B9u + 0x7F4A7C15u;
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  v[i] = (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
}

__global__ void __launch_bounds__(kWtThreads) wt_sumsq_kernel(int32_t n, const float *__restrict__ u,
                                                             double *__restrict__ part) {
  __shared__ double red[kWtThreads / 32];
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a += (double)u[i] * u[i];
  const double b = block_sum<kWtThreads>(a, red);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void wt_total_kernel(int nb, const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double red[4];
  double a = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) a += part[k];
  const double b = block_sum<128>(a, red);
  if (threadIdx.x == 0) *out = b;
}

__global__ void wt_normalise_kernel(int32_t n, const float *__restrict__ u, const double *__restrict__ ss,
                                    float *__restrict__ v) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double q = *ss;
  v[i] = q > 0.0 ? (float)(u[i] / sqrt(q)) : 0.0f;
}

// window w of a rollout: r = (Tref + Tmax y - T*) / T* at the window's end y,
// block sums of r^p into part, and Lam += p r^(p-1) Tmax / (n T*)
__global__ void __launch_bounds__(kWtThreads) wt_rollout_loss_kernel(int32_t n, const float *__restrict__ y,
                                                                    const double *__restrict__ Tt, double Tref,
                                                                    double Tmax, int pw, float *__restrict__ Lam,
                                                                    double *__restrict__ part) {
  __shared__ double red[kWtThreads / 32];
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double rp = 0.0;
  if (i < n) {
    const double t = Tt[i];
    const double r = (fma(Tmax, (double)y[i], Tref) - t) / t;
    double rq = r;
    for (int k = 2; k < pw; ++k) rq *= r;
    rp = rq * r;
    Lam[i] += (float)(pw * rq * Tmax / ((double)n * t));
  }
  const double b = block_sum<kWtThreads>(rp, red);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// out = a + b (the next window's start), out = c x + y (the VJP input), x += y
__global__ void wt_add_kernel(int32_t n, const float *__restrict__ a, const float *__restrict__ b,
                              float *__restrict__ out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + b[i];
}
__global__ void wt_axpy_kernel(int32_t n, float c, const float *__restrict__ x, const float *__restrict__ y,
                               float *__restrict__ out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = fmaf(c, x[i], y[i]);
}

__global__ void wt_end_kernel(int64_t n, const double *__restrict__ T0, const float *__restrict__ zs, double Tmax,
                              double *__restrict__ T1) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) T1[i] = fma(Tmax, (double)zs[i], T0[i]);
}

}  // namespace

cudaError_t wt_stages(Ctx &c, int s, const WtCoef &k, const float *y0, const WtTab &t) {
  if (c.n == 0) return cudaSuccess;
  const int32_t n = (int32_t)c.n;
  const float th = (float)(c.p.Tref_K / c.p.Tmax_K);
  for (int j = 1; j <= s; ++j) {
    wt_stage_kernel<<<wblk(n), kWtThreads, 0, c.stream>>>(
        n, c.nbr, c.cnt, th, y0, j >= 2 ? t.z[j - 1] : nullptr, j >= 3 ? t.z[j - 2] : nullptr,
        j >= 2 ? t.F[1] : nullptr, k.nu[j], k.kap[j], k.a[j], k.g[j], const_cast<float *>(t.F[j]),
        const_cast<float *>(t.z[j]));
  }
  return cudaGetLastError();
}

cudaError_t wt_backward(Ctx &c, int s, const WtCoef &k, const float *y0, const WtTab &t, const double *T0,
                        const double *T1, int loss_power, double *lpart, double *dpart, double tauK,
                        const float *c0, float *gc, float *gd, float *loss) {
  if (c.n == 0) return cudaSuccess;
  const int32_t n = (int32_t)c.n;
  const float th = (float)(c.p.Tref_K / c.p.Tmax_K);
  for (int j = 1; j < s; ++j) {
    cudaError_t e = cudaMemsetAsync(const_cast<float *>(t.lam[j]), 0, sizeof(float) * n, c.stream);
    if (e != cudaSuccess) return e;
  }
  const unsigned nbl = wblk(n);
  wt_loss_kernel<<<nbl, kWtThreads, 0, c.stream>>>(n, t.z[s], T0, T1, c.p.Tmax_K, loss_power,
                                                   const_cast<float *>(t.lam[s]), lpart);
  for (int j = s; j >= 2; --j)
    wt_adjoint_kernel<<<wblk(n), kWtThreads, 0, c.stream>>>(
        n, c.nbr, c.cnt, th, y0, t.z[j - 1], t.lam[j], 1.0f - k.nu[j] - k.kap[j], k.a[j], k.nu[j],
        const_cast<float *>(t.lam[j - 1]), j >= 3 ? const_cast<float *>(t.lam[j - 2]) : nullptr);
  const unsigned nbd = std::min<unsigned>(wblk(n), kWtDotBlocks);
  wt_dots_kernel<<<dim3(nbd, s), kWtThreads, 0, c.stream>>>(n, t, dpart);
  wt_final_kernel<<<4 * (s + 1) + 1, 128, 0, c.stream>>>(s, (int)nbd, dpart, (int)nbl, lpart, tauK, 1.0 / n, c0,
                                                         gc, gd, loss);
  return cudaGetLastError();
}

cudaError_t wt_rollout(Ctx &c, int s, const WtCoef &k, int nwin, const float *const *y0, const WtTab *t,
                       const double *const *Tt, float *const *lam, float *Lam, float *mu, float *gs, float *tmp,
                       const float *zero, int loss_power, double *lpart, double *dpart, double tauK,
                       const float *c0, float *gc, float *gd, float *loss) {
  if (c.n == 0) return cudaSuccess;
  const int32_t n = (int32_t)c.n;
  const float th = (float)(c.p.Tref_K / c.p.Tmax_K);
  const unsigned nb = wblk(n), nbl = wblk(n);
  const unsigned nbd = std::min<unsigned>(wblk(n), kWtDotBlocks);
  cudaError_t e = cudaMemsetAsync(Lam, 0, sizeof(float) * n, c.stream);
  for (int w = nwin - 1; w >= 0 && e == cudaSuccess; --w) {
    // the loss of window w at its end y0[w + 1] seeds Lam
    wt_rollout_loss_kernel<<<nbl, kWtThreads, 0, c.stream>>>(n, y0[w + 1], Tt[w], c.p.Tref_K, c.p.Tmax_K,
                                                             loss_power, Lam, lpart + (size_t)w * nbl);
    WtTab tw = t[w];
    for (int j = 1; j <= s; ++j) tw.lam[j] = lam[j];
    e = cudaMemcpyAsync(lam[s], Lam, sizeof(float) * n, cudaMemcpyDeviceToDevice, c.stream);
    for (int j = 1; j < s && e == cudaSuccess; ++j) e = cudaMemsetAsync(lam[j], 0, sizeof(float) * n, c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(mu, 0, sizeof(float) * n, c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(gs, 0, sizeof(float) * n, c.stream);
    if (e != cudaSuccess) break;
    for (int j = s; j >= 2; --j)
      wt_adjoint_kernel<<<nb, kWtThreads, 0, c.stream>>>(n, c.nbr, c.cnt, th, y0[w], tw.z[j - 1], lam[j],
                                                          1.0f - k.nu[j] - k.kap[j], k.a[j], k.nu[j], lam[j - 1],
                                                          j >= 3 ? lam[j - 2] : nullptr, k.g[j], mu, gs);
    wt_dots_kernel<<<dim3(nbd, s), kWtThreads, 0, c.stream>>>(n, tw, dpart, w < nwin - 1 ? 1 : 0);
    // mu += J(Y_0)^T (a_1 lam_1 + gs): the adjoint kernel at Y_0 (zero change)
    wt_axpy_kernel<<<nb, kWtThreads, 0, c.stream>>>(n, k.a[1], lam[1], gs, tmp);
    wt_adjoint_kernel<<<nb, kWtThreads, 0, c.stream>>>(n, c.nbr, c.cnt, th, y0[w], zero, tmp, 0.0f, 1.0f, 0.0f, mu,
                                                        nullptr);
    // the window-start adjoint: Lam (the end's) + mu
    wt_add_kernel<<<nb, kWtThreads, 0, c.stream>>>(n, Lam, mu, Lam);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  wt_final_kernel<<<4 * (s + 1) + 1, 128, 0, c.stream>>>(s, (int)nbd, dpart, (int)(nbl * nwin), lpart, tauK,
                                                         1.0 / n, c0, gc, gd, loss);
  return cudaGetLastError();
}

cudaError_t wt_next_start(Ctx &c, const float *y0, const float *zs, float *y1) {
  if (c.n > 0) wt_add_kernel<<<wblk(c.n), kWtThreads, 0, c.stream>>>((int32_t)c.n, y0, zs, y1);
  return cudaGetLastError();
}

size_t wt_dot_partials(int64_t n, int s) {
  const unsigned nbd = std::min<unsigned>(wblk(n > 0 ? n : 1), kWtDotBlocks);
  return (size_t)4 * (s + 1) * nbd;
}

size_t wt_loss_partials(int64_t n) { return wblk(n > 0 ? n : 1); }

cudaError_t wt_adam(cudaStream_t st, int np, float *p, float *m, float *v, const float *g, float lr, int t) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  wt_adam_kernel<<<(np + 127) / 128, 128, 0, st>>>(np, p, m, v, g, lr, b1, b2, 1e-12f, c1, c2);
  return cudaGetLastError();
}

cudaError_t wt_power(Ctx &c, const float *y, const float *zero, float *v, float *u, double *part, double *ss,
                     int iters) {
  if (c.n == 0) return cudaSuccess;
  const int32_t n = (int32_t)c.n;
  const float th = (float)(c.p.Tref_K / c.p.Tmax_K);
  const unsigned nbd = std::min<unsigned>(wblk(n), kWtDotBlocks);
  wt_seed_kernel<<<wblk(n), kWtThreads, 0, c.stream>>>(n, u);
  for (int it = 0; it <= iters; ++it) {
    // v = u / |u|; then u = J(y)^T v (the adjoint kernel with lam_{j-1} = u zeroed,
    // c1 = 0, a = 1), so that |u| -> |lambda_max| as the iteration converges
    wt_sumsq_kernel<<<nbd, kWtThreads, 0, c.stream>>>(n, u, part);
    wt_total_kernel<<<1, 128, 0, c.stream>>>((int)nbd, part, ss);
    if (it == iters) break;
    wt_normalise_kernel<<<wblk(n), kWtThreads, 0, c.stream>>>(n, u, ss, v);
    cudaError_t e = cudaMemsetAsync(u, 0, sizeof(float) * n, c.stream);
    if (e != cudaSuccess) return e;
    wt_adjoint_kernel<<<wblk(n), kWtThreads, 0, c.stream>>>(n, c.nbr, c.cnt, th, y, zero, v, 0.0f, 1.0f, 0.0f, u,
                                                           nullptr);
  }
  return cudaGetLastError();
}

cudaError_t wt_end(Ctx &c, const double *T0, const float *zs, double *T1) {
  if (c.n > 0) wt_end_kernel<<<wblk(c.n), kWtThreads, 0, c.stream>>>(c.n, T0, zs, c.p.Tmax_K, T1);
  return cudaGetLastError();
}

}  // namespace ehc
