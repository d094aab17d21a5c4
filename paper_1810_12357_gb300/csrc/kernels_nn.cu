// kernels_nn.cu -- the learned window propagator: forward, backward, Adam,
// and the a-posteriori residual of a window.
//
// The network replaces n_w explicit substeps of Eq. HeatTransport (pair-flux
// part) on the context's neighbour graph.  With delta = (T - Tref)/Tmax (the
// substep mirror), D_ij = (delta_j - delta_i)/sigma, q = D^2/(1+D^2),
// s = theta_i + theta_j, hidden width H:
//   h_i    = sum_j D_ij relu(W1 [q, s] + b1)                          (layer 1, R^H)
//   phi_ij = D_ij (c0 + w . relu(W2 [q, s] + b2)) + u . (h_j - h_i)   (layer 2)
//   T^_i   = T_i + sigma Tmax kappa sum_j phi_ij,   kappa = n_w dt K
// Every pair term is odd under i <-> j, so the pair fluxes conserve sum_i T_i.
// Weights are held in BF16 for the forward (FP32 master copy for training), the
// hidden vectors h in BF16, all arithmetic and accumulation in FP32.
// Parameter layout (8H + 1): [W1 (H x 2) | b1 | W2 (H x 2) | b2 | w | u | c0].
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr int kNnThreads = 256;

struct NnScal {
  float inv_sigma, th2;     // 1/sigma, 2 Tref/Tmax
  double scale;             // sigma Tmax kappa
  double Tref, invTmax;
};

template <int H>
struct W {
  float W1[H][2], b1[H], W2[H][2], b2[H], w[H], u[H], c0;
};

template <int H>
__device__ __forceinline__ void load_w(const __nv_bfloat16 *__restrict__ pb, W<H> &s) {
  float *dst = reinterpret_cast<float *>(&s);
  for (int k = threadIdx.x; k < 8 * H + 1; k += blockDim.x) dst[k] = __bfloat162float(pb[k]);
}

__device__ __forceinline__ void edge_feat(float di, float dj, const NnScal &c, float &D, float &q, float &s) {
  D = (dj - di) * c.inv_sigma;
  const float D2 = D * D;
  q = D2 / (1.0f + D2);
  s = c.th2 + di + dj;
}

// gather the sorted-order state of the window from caller-order arrays
__global__ void nn_gather_kernel(int64_t n, const int32_t *__restrict__ inv, const double *__restrict__ Tin,
                                 const double *__restrict__ Ttar, double Tref, double invTmax,
                                 double *__restrict__ Ts, double *__restrict__ Ttar_s, float *__restrict__ dmir) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int64_t s = inv ? inv[o] : o;
  const double t = Tin[o];
  Ts[s] = t;
  if (Ttar) Ttar_s[s] = Ttar[o];
  dmir[s] = (float)((t - Tref) * invTmax);
}

template <int H>
__global__ void __launch_bounds__(kNnThreads) nn_layer1_kernel(int32_t n, const int32_t *__restrict__ nbr,
                                                               const uint8_t *__restrict__ cnt,
                                                               const float *__restrict__ dm,
                                                               const __nv_bfloat16 *__restrict__ pb, NnScal c,
                                                               __nv_bfloat16 *__restrict__ hout) {
  __shared__ W<H> w;
  load_w<H>(pb, w);
  __syncthreads();
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float di = dm[i];
  float h[H];
#pragma unroll
  for (int k = 0; k < H; ++k) h[k] = 0.0f;
  const int ci = cnt[i];
  for (int e = 0; e < ci; ++e) {
    const float dj = __ldg(dm + __ldg(nbr + (int64_t)e * n + i));
    float D, q, s;
    edge_feat(di, dj, c, D, q, s);
#pragma unroll
    for (int k = 0; k < H; ++k) h[k] = fmaf(D, fmaxf(fmaf(w.W1[k][0], q, fmaf(w.W1[k][1], s, w.b1[k])), 0.0f), h[k]);
  }
#pragma unroll
  for (int k = 0; k < H; ++k) hout[(int64_t)i * H + k] = __float2bfloat16(h[k]);
}

// block reduction of NV per-thread values into part[blockIdx.x][NV] (fixed order)
template <int NV>
__device__ __forceinline__ void block_reduce_store(float (&v)[NV], float *__restrict__ part) {
  __shared__ float red[kNnThreads / 32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[wid][k] = x;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    float x = 0.0f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) x += red[q][k];
    part[(int64_t)blockIdx.x * NV + k] = x;
  }
}

// Layer 2.  Inference: T^ into Tout (FP64) and its mirror into dm_out.
// Training (Ttar != null): residual, dL/dT^, the layer-2 parameter gradients and
// the loss, reduced per block into part[block][5H+2] = [c0 | w | W2 | b2 | u | loss].
template <int H, bool TRAIN>
__global__ void __launch_bounds__(kNnThreads) nn_layer2_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt, const float *__restrict__ dm,
    const __nv_bfloat16 *__restrict__ hb, const __nv_bfloat16 *__restrict__ pb, NnScal c,
    const double *__restrict__ Tin, double *__restrict__ Tout, float *__restrict__ dm_out,
    const double *__restrict__ Ttar, float inv_ts, float gscale, float *__restrict__ gphi,
    float *__restrict__ part) {
  constexpr int NV = 5 * H + 2;
  __shared__ W<H> w;
  load_w<H>(pb, w);
  __syncthreads();
  float acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0f;
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float di = dm[i];
    const int ci = cnt[i];
    float sumD = 0.0f, Fw = 0.0f;
    float hs[H], dw[H], dW2q[H], dW2s[H], db2[H];
#pragma unroll
    for (int k = 0; k < H; ++k) hs[k] = dw[k] = dW2q[k] = dW2s[k] = db2[k] = 0.0f;
    for (int e = 0; e < ci; ++e) {
      const int32_t j = __ldg(nbr + (int64_t)e * n + i);
      const float dj = __ldg(dm + j);
      float D, q, s;
      edge_feat(di, dj, c, D, q, s);
      sumD += D;
      float wa = 0.0f;
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const float z = fmaf(w.W2[k][0], q, fmaf(w.W2[k][1], s, w.b2[k]));
        const float a = fmaxf(z, 0.0f);
        wa = fmaf(w.w[k], a, wa);
        if (TRAIN) {
          dw[k] = fmaf(D, a, dw[k]);
          const float m = z > 0.0f ? D * w.w[k] : 0.0f;
          dW2q[k] = fmaf(m, q, dW2q[k]);
          dW2s[k] = fmaf(m, s, dW2s[k]);
          db2[k] += m;
        }
      }
      Fw = fmaf(D, wa, Fw);
#pragma unroll
      for (int k = 0; k < H; ++k) hs[k] += __bfloat162float(hb[(int64_t)j * H + k]);
    }
    // u . (sum_j h_j - deg h_i)
    float Fu = 0.0f;
    float hdiff[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
      hdiff[k] = hs[k] - (float)ci * __bfloat162float(hb[(int64_t)i * H + k]);
      Fu = fmaf(w.u[k], hdiff[k], Fu);
    }
    const float F = fmaf(w.c0, sumD, Fw) + Fu;
    const double That = Tin[i] + c.scale * (double)F;
    if (!TRAIN) {
      Tout[i] = That;
      dm_out[i] = (float)((That - c.Tref) * c.invTmax);
    } else {
      const float r = (float)((That - Ttar[i]) * (double)inv_ts);
      const float g = gscale * r;        // dL/dphi for the edges of atom i
      gphi[i] = g;
      acc[0] = g * sumD;
#pragma unroll
      for (int k = 0; k < H; ++k) {
        acc[1 + k] = g * dw[k];
        acc[1 + H + 2 * k] = g * dW2q[k];
        acc[1 + H + 2 * k + 1] = g * dW2s[k];
        acc[1 + 3 * H + k] = g * db2[k];
        acc[1 + 4 * H + k] = g * hdiff[k];
      }
      acc[NV - 1] = r * r;
    }
  }
  if (TRAIN) block_reduce_store<NV>(acc, part);
}

// Layer-1 gradients: dL/dh_m = u * S_m with S_m = sum_{i in N(m)} gphi_i - deg(m) gphi_m;
// part[block][3H] = [W1 (H x 2) | b1]
template <int H>
__global__ void __launch_bounds__(kNnThreads) nn_back1_kernel(int32_t n, const int32_t *__restrict__ nbr,
                                                              const uint8_t *__restrict__ cnt,
                                                              const float *__restrict__ dm,
                                                              const __nv_bfloat16 *__restrict__ pb, NnScal c,
                                                              const float *__restrict__ gphi,
                                                              float *__restrict__ part) {
  constexpr int NV = 3 * H;
  __shared__ W<H> w;
  load_w<H>(pb, w);
  __syncthreads();
  float acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0f;
  const int32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n) {
    const float dmm = dm[m];
    const int cm = cnt[m];
    float S = -(float)cm * gphi[m];
    for (int e = 0; e < cm; ++e) S += __ldg(gphi + __ldg(nbr + (int64_t)e * n + m));
    for (int e = 0; e < cm; ++e) {
      const float dj = __ldg(dm + __ldg(nbr + (int64_t)e * n + m));
      float D, q, s;
      edge_feat(dmm, dj, c, D, q, s);
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const float z = fmaf(w.W1[k][0], q, fmaf(w.W1[k][1], s, w.b1[k]));
        const float g = z > 0.0f ? S * w.u[k] * D : 0.0f;
        acc[2 * k] = fmaf(g, q, acc[2 * k]);
        acc[2 * k + 1] = fmaf(g, s, acc[2 * k + 1]);
        acc[2 * H + k] += g;
      }
    }
  }
  block_reduce_store<NV>(acc, part);
}

// sum the block partials (fixed order) into the gradient in parameter order,
// and the loss; one block
template <int H>
__global__ void nn_grad_final_kernel(int nb, const float *__restrict__ p2, const float *__restrict__ p1,
                                     float *__restrict__ grad, float *__restrict__ loss, float inv_n) {
  constexpr int NV2 = 5 * H + 2, NV1 = 3 * H, NP = 8 * H + 1;
  for (int k = threadIdx.x; k < NP + 1; k += blockDim.x) {
    // map parameter k to its partial slot
    int src = -1, which = 0;
    if (k < 2 * H) { which = 1; src = k; }                       // W1
    else if (k < 3 * H) { which = 1; src = 2 * H + (k - 2 * H); }  // b1
    else if (k < 5 * H) { which = 2; src = 1 + H + (k - 3 * H); }  // W2
    else if (k < 6 * H) { which = 2; src = 1 + 3 * H + (k - 5 * H); }  // b2
    else if (k < 7 * H) { which = 2; src = 1 + (k - 6 * H); }      // w
    else if (k < 8 * H) { which = 2; src = 1 + 4 * H + (k - 7 * H); }  // u
    else if (k == 8 * H) { which = 2; src = 0; }                   // c0
    else { which = 2; src = NV2 - 1; }                             // loss
    double x = 0.0;
    for (int b = 0; b < nb; ++b) x += which == 1 ? (double)p1[(int64_t)b * NV1 + src] : (double)p2[(int64_t)b * NV2 + src];
    if (k < NP) grad[k] = (float)x;
    else *loss = (float)(x * inv_n);
  }
}

// Adam on the FP32 master weights; refreshes the BF16 copy
__global__ void nn_adam_kernel(int np, float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                               const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1,
                               float c2, __nv_bfloat16 *__restrict__ pb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.0f - b1) * gk;
  const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  p[k] = pk;
  pb[k] = __float2bfloat16(pk);
}

__global__ void nn_to_bf16_kernel(int np, const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < np) pb[k] = __float2bfloat16(p[k]);
}

// a-posteriori residual of a window of length tau: with R the right-hand side of
// Eq. HeatTransport (pair flux and coupling) at the old and the predicted state,
// rho_i = |T^_i - T_i - tau (R(T)_i + R(T^)_i)/2| / max(1 K, 1e-3 T_i); block maxima
__global__ void __launch_bounds__(kNnThreads) nn_residual_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt, const float *__restrict__ d0,
    const float *__restrict__ d1, const double *__restrict__ T0, const double *__restrict__ T1,
    const float *__restrict__ uTl, const StepCoef *__restrict__ cf, double tau, float *__restrict__ part) {
  __shared__ float red[kNnThreads / 32];
  float rho = 0.0f;
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float th = cf->th_ref;
    const float a0 = d0[i], a1 = d1[i];
    float F0 = 0.0f, F1 = 0.0f;
    const int ci = cnt[i];
    for (int e = 0; e < ci; ++e) {
      const int32_t j = __ldg(nbr + (int64_t)e * n + i);
      // f(a, b) = Delta cosh(Delta) - P sinh(Delta), Taylor series to Delta^10
      const float b0 = __ldg(d0 + j), b1 = __ldg(d1 + j);
      for (int t = 0; t < 2; ++t) {
        const float a = t ? a1 : a0, b = t ? b1 : b0;
        const float D = b - a, x = D * D;
        float S = fmaf(x, 2.5052108e-08f, 2.7557319e-06f);
        S = fmaf(x, S, 1.9841270e-04f);
        S = fmaf(x, S, 8.3333333e-03f);
        S = fmaf(x, S, 1.6666667e-01f);
        S = fmaf(x, S, 1.0f);
        float C = fmaf(x, 2.7557319e-07f, 2.4801587e-05f);
        C = fmaf(x, C, 1.3888889e-03f);
        C = fmaf(x, C, 4.1666667e-02f);
        C = fmaf(x, C, 0.5f);
        C = fmaf(x, C, 1.0f);
        const float ta = th + a, tb = th + b;
        const float P = fmaf(-2.0f * ta, tb, ta + tb);
        const float f = D * fmaf(-P, S, C);
        if (t) F1 += f;
        else F0 += f;
      }
    }
    // R = Tmax K F - (G/C_e)(T - T_l); dtTK / dt = Tmax K, dtcG / dt = G / C_e
    const double TK = cf->dtTK / cf->dt, cG = cf->dtcG / cf->dt;
    const float ui = uTl[i];
    const bool chi = ui == ui;
    const double Tl = chi ? cf->Tref - (double)ui : 0.0;
    const double R0 = TK * (double)F0 - (chi ? cG * (T0[i] - Tl) : 0.0);
    const double R1 = TK * (double)F1 - (chi ? cG * (T1[i] - Tl) : 0.0);
    const double res = fabs(T1[i] - T0[i] - 0.5 * tau * (R0 + R1));
    const double den = fmax(1.0, 1e-3 * T0[i]);
    rho = (float)(res / den);
    if (!(rho == rho)) rho = 3.0e38f;
  }
  for (int o = 16; o > 0; o >>= 1) rho = fmaxf(rho, __shfl_down_sync(0xffffffffu, rho, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rho;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
    part[blockIdx.x] = r;
  }
}

__global__ void max_final_kernel(int nb, const float *__restrict__ part, float *__restrict__ out) {
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

// electron-phonon coupling over a window of n_w substeps, applied after the
// predicted flux: T -= f (T0 - T_l) with f = 1 - (1 - dt G/C_e)^n_w; the
// decrement is kept in dTc and handed to the lattice ledger A (Eq. RateExchange)
// only if the window is accepted
__global__ void nn_couple_window_kernel(int64_t n, const double *__restrict__ T0, double *__restrict__ T1,
                                        float *__restrict__ d1, const float *__restrict__ uTl,
                                        double *__restrict__ dTc, double f, double Tref, double invTmax) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float ui = uTl[s];
  if (!(ui == ui)) {
    dTc[s] = 0.0;
    return;
  }
  const double dT = f * (T0[s] - (Tref - (double)ui));
  const double t1 = T1[s] - dT;
  T1[s] = t1;
  d1[s] = (float)((t1 - Tref) * invTmax);
  dTc[s] = dT;
}

__global__ void nn_accept_kernel(int64_t n, const double *__restrict__ dTc, double VC, double *__restrict__ A) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s < n) A[s] += VC * dTc[s];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers (host side of ehc_nn_*)

cudaError_t nn_couple_window(Ctx &c, const double *T0, double *T1, float *d1, double *dTc, int n_w) {
  if (c.n == 0) return cudaSuccess;
  const double f = 1.0 - std::pow(1.0 - c.p.dt_sub_fs * c.cG, (double)n_w);
  nn_couple_window_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(c.n, T0, T1, d1, c.uTl, dTc, f, c.p.Tref_K,
                                                                1.0 / c.p.Tmax_K);
  return cudaGetLastError();
}

cudaError_t nn_accept(Ctx &c, const double *dTc) {
  if (c.n == 0) return cudaSuccess;
  nn_accept_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(c.n, dTc, c.VC, c.A);
  return cudaGetLastError();
}

int nn_blocks(int64_t n) { return (int)nblk(n, kNnThreads); }

// sorted == true: Tin (and Ttar) are already in the context's sorted order
cudaError_t nn_gather(Ctx &c, const double *Tin, const double *Ttar, double *Ts, double *Ttar_s, float *dm,
                      bool sorted) {
  if (c.n > 0)
    nn_gather_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(c.n, sorted ? nullptr : c.inv_perm[c.cur_inv], Tin, Ttar,
                                                           c.p.Tref_K, 1.0 / c.p.Tmax_K, Ts, Ttar_s, dm);
  return cudaGetLastError();
}

static NnScal make_scal(const Ctx &c, double sigma, int n_w) {
  NnScal s;
  s.inv_sigma = (float)(1.0 / sigma);
  s.th2 = (float)(2.0 * c.p.Tref_K / c.p.Tmax_K);
  s.scale = sigma * c.p.Tmax_K * (double)n_w * c.p.dt_sub_fs * c.K;
  s.Tref = c.p.Tref_K;
  s.invTmax = 1.0 / c.p.Tmax_K;
  return s;
}

cudaError_t nn_forward(Ctx &c, int H, const __nv_bfloat16 *pb, double sigma, int n_w, const float *dm,
                       __nv_bfloat16 *h, const double *Tin, double *Tout, float *dm_out) {
  if (c.n == 0) return cudaSuccess;
  const NnScal s = make_scal(c, sigma, n_w);
  const int32_t n = (int32_t)c.n;
  const unsigned nb = nblk(n, kNnThreads);
  if (H == 8) {
    nn_layer1_kernel<8><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, pb, s, h);
    nn_layer2_kernel<8, false><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, h, pb, s, Tin, Tout, dm_out,
                                                                nullptr, 0.f, 0.f, nullptr, nullptr);
  } else {
    nn_layer1_kernel<16><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, pb, s, h);
    nn_layer2_kernel<16, false><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, h, pb, s, Tin, Tout, dm_out,
                                                                 nullptr, 0.f, 0.f, nullptr, nullptr);
  }
  return cudaGetLastError();
}

// forward + backward of one window; grad (8H+1 floats) and loss on the device
cudaError_t nn_grad(Ctx &c, int H, const __nv_bfloat16 *pb, double sigma, int n_w, const float *dm,
                    __nv_bfloat16 *h, const double *Tin, const double *Ttar, float *gphi, float *p2, float *p1,
                    float *grad, float *loss) {
  if (c.n == 0) return cudaSuccess;
  const NnScal s = make_scal(c, sigma, n_w);
  const int32_t n = (int32_t)c.n;
  const unsigned nb = nblk(n, kNnThreads);
  const double Ts = sigma * c.p.Tmax_K;
  const float inv_ts = (float)(1.0 / Ts);
  // dL/dphi_ij = dL/dT^_i * scale = 2 r_i / (N Ts) * scale
  const float gscale = (float)(2.0 / ((double)n * Ts) * s.scale);
  if (H == 8) {
    nn_layer1_kernel<8><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, pb, s, h);
    nn_layer2_kernel<8, true><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, h, pb, s, Tin, nullptr, nullptr,
                                                               Ttar, inv_ts, gscale, gphi, p2);
    nn_back1_kernel<8><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, pb, s, gphi, p1);
    nn_grad_final_kernel<8><<<1, 128, 0, c.stream>>>((int)nb, p2, p1, grad, loss, 1.0f / (float)n);
  } else {
    nn_layer1_kernel<16><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, pb, s, h);
    nn_layer2_kernel<16, true><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, h, pb, s, Tin, nullptr,
                                                                nullptr, Ttar, inv_ts, gscale, gphi, p2);
    nn_back1_kernel<16><<<nb, kNnThreads, 0, c.stream>>>(n, c.nbr, c.cnt, dm, pb, s, gphi, p1);
    nn_grad_final_kernel<16><<<1, 256, 0, c.stream>>>((int)nb, p2, p1, grad, loss, 1.0f / (float)n);
  }
  return cudaGetLastError();
}

cudaError_t nn_adam(cudaStream_t st, int np, float *p, float *m, float *v, const float *g, float lr, int t,
                    __nv_bfloat16 *pb) {
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.0f, c2 = 1.0f;
  for (int k = 0; k < t; ++k) {
    c1 *= b1;
    c2 *= b2;
  }
  nn_adam_kernel<<<1, 256, 0, st>>>(np, p, m, v, g, lr, b1, b2, 1e-8f, 1.0f - c1, 1.0f - c2, pb);
  return cudaGetLastError();
}

cudaError_t nn_params_to_bf16(cudaStream_t st, int np, const float *p, __nv_bfloat16 *pb) {
  nn_to_bf16_kernel<<<1, 256, 0, st>>>(np, p, pb);
  return cudaGetLastError();
}

cudaError_t nn_residual(Ctx &c, const float *d0, const float *d1, const double *T0, const double *T1, double tau,
                        float *part, float *out) {
  if (c.n == 0) return cudaSuccess;
  const unsigned nb = nblk(c.n, kNnThreads);
  nn_residual_kernel<<<nb, kNnThreads, 0, c.stream>>>((int32_t)c.n, c.nbr, c.cnt, d0, d1, T0, T1, c.uTl, c.coef,
                                                      tau, part);
  max_final_kernel<<<1, 256, 0, c.stream>>>((int)nb, part, out);
  return cudaGetLastError();
}

}  // namespace ehc
