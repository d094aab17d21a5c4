// kernels_couple.cu -- once-per-MD-step hand-over of the exchanged energy to
// the atoms, the free-flight drift, and the Philox4x32-10 generator.
//
// Energy balance (Eqs. RateExchange, WorkDone, Xi): during the substeps the
// electrons of atom i gave up A_i = dt sum_n G V_atom (T_i - T_l,i).  The
// damping force xi_i m v_i of Eq. Motion, with xi_i of Eq. Xi, integrated over
// the MD step scales the velocity by s with s^2 = (K_i + A_i) / K_i, which
// moves exactly A_i into the atom's kinetic energy K_i.  The Langevin variant
// first applies friction e^{-g dt} and a Gaussian random force of variance
// k_B T_e,i (1 - e^{-2 g dt}) / m (g = G V_atom / (3 k_B)), then rescales to the
// same kinetic energy K_i + A_i, so the hand-over stays exact.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr double kMVV = 1.66053906660e-27 * 1.0e10 / 1.602176634e-19;  // amu (A/fs)^2 -> eV
constexpr double kKB = 8.617333262e-5;
constexpr double kEVJ = 1.602176634e-19;   // J per eV

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplications (high and low halves) with Weyl-sequence key increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

// counter (id lo, id hi, step lo, step hi), key (seed lo, seed hi); the top
// 24 bits of each output word give u = (x + 1/2) 2^-24 in (0, 1), exact in
// single precision; Box-Muller in single precision.
__device__ __forceinline__ void gauss3(uint64_t id, uint64_t step, uint64_t seed, float g[3]) {
  const uint4 r = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step,
                                           (uint32_t)(step >> 32)),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float s = 5.9604644775390625e-08f;  // 2^-24
  const float u0 = ((float)(r.x >> 8) + 0.5f) * s, u1 = ((float)(r.y >> 8) + 0.5f) * s;
  const float u2 = ((float)(r.z >> 8) + 0.5f) * s, u3 = ((float)(r.w >> 8) + 0.5f) * s;
  const float r1 = sqrtf(-2.0f * logf(u0));
  const float r2 = sqrtf(-2.0f * logf(u2));
  float sn, cs;
  sincospif(2.0f * u1, &sn, &cs);
  g[0] = r1 * cs;
  g[1] = r1 * sn;
  g[2] = r2 * cospif(2.0f * u3);
}

// s = sqrt(target / Kw) without an FP64 division or square root: Newton's
// method for f(y) = Kw y^2 - target, started from the single-precision root and
// stepped twice in FP64 with a single-precision 1 / f'(y0) (each step squares
// the relative error, 1e-7 -> 1e-14 -> rounding).  Outside the normal
// single-precision range the plain FP64 expression is used.
__device__ __forceinline__ double scale_root(double target, double Kw) {
  if (!(target > 1.0e-30 && target < 1.0e30 && Kw > 1.0e-30 && Kw < 1.0e30)) return sqrt(target / Kw);
  const float kf = (float)Kw;
  const float yf = sqrtf((float)target / kf);
  const double c = (double)(0.5f / (kf * yf));   // ~ 1 / (2 Kw y)
  double y = (double)yf;
#pragma unroll
  for (int it = 0; it < 2; ++it) y = fma(fma(-Kw * y, y, target), c, y);
  return y;
}

__global__ void couple_kernel(int64_t n, const int32_t *__restrict__ perm, const int8_t *__restrict__ type_s,
                              MassTable mt, double kv, double kv0, const double *__restrict__ Tl,
                              double *__restrict__ A,
                              double *__restrict__ T, double *__restrict__ v, double *__restrict__ dKE,
                              int mode, int frozen, uint64_t seed, uint64_t md_step, double e1, double inv_VC,
                              unsigned long long *__restrict__ n_stopped, double thc, double inv_Tmax,
                              double stop_f, double stop_ecut) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double Ai = A[s];
  A[s] = 0.0;
  if (!(Tl[s] >= 0.0)) {
    dKE[s] = 0.0;
    return;
  }
  if (frozen) {
    dKE[s] = Ai;
    return;
  }
  const int64_t o = perm[s];
  const int ty = type_s[s];
  const double m = mt.m[ty];
  double *vi = v + 3 * o;
  const double v0 = vi[0], v1 = vi[1], v2 = vi[2];
  const double K0 = 0.5 * m * (v0 * v0 + v1 * v1 + v2 * v2) * kMVV;
  double target = K0 + Ai;
  // electronic stopping above the cut: the friction's loss over the MD step
  const bool slowed = stop_f > 0.0 && K0 > stop_ecut;
  if (slowed) target -= K0 * stop_f;
  if (target < 0.0) {
    target = 0.0;
    atomicAdd(n_stopped, 1ull);
  }
  double w0 = v0, w1 = v1, w2 = v2;
  if (mode == 1) {
    float g[3];
    gauss3((uint64_t)o, md_step, seed, g);
    // noise amplitude in single precision (it multiplies a single-precision normal)
    // variance factor k_B (1 - e^{-2 g dt}) / (m kMVV) = kv / (m kMVV), for type 0 from the host
    const double cv = (ty == 0) ? kv0 : kv / (m * kMVV);
    const float sig = sqrtf((float)(cv * T[s]));
    w0 = v0 * e1 + (double)(sig * g[0]);
    w1 = v1 * e1 + (double)(sig * g[1]);
    w2 = v2 * e1 + (double)(sig * g[2]);
  }
  const double Kw = 0.5 * m * (w0 * w0 + w1 * w1 + w2 * w2) * kMVV;
  const double sc = (Kw > 0.0 && target > 0.0) ? scale_root(target, Kw) : 0.0;
  vi[0] = w0 * sc;
  vi[1] = w1 * sc;
  vi[2] = w2 * sc;
  // the new kinetic energy is the target up to the rounding of the scaling
  const double d = target - K0;
  dKE[s] = d;
  if (target == 0.0 || slowed) {
    // the unpaid part (and the stopping loss) goes to the atom's electrons: T += dE / (V_atom C_e), or in
    // the LOCAL form (inv_Tmax > 0) u += dE / (V_atom gamma Tmax^2) with inv_VC that factor
    if (inv_Tmax > 0.0) T[s] = ue_inv(ue_of(T[s] * inv_Tmax, thc) + (Ai - d) * inv_VC, thc) / inv_Tmax;
    else T[s] += (Ai - d) * inv_VC;
  }
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;
}

__global__ void sum_partial(int64_t n, const double *__restrict__ x, double *__restrict__ part) {
  __shared__ double sh[32];
  double a = 0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    a += x[s];
  double r = block_sum(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void sum_final_accumulate(int nb, const double *__restrict__ part, double *__restrict__ acc) {
  __shared__ double sh[32];
  double a = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[b];
  double r = block_sum(a, sh);
  if (threadIdx.x == 0) *acc += r;
}

// sign and ordering tests of doubles on the integer pipes: for y >= 0 the bit
// patterns order like the values
__device__ __forceinline__ bool neg_bits(double y) { return __double_as_longlong(y) < 0; }
__device__ __forceinline__ bool ge_bits(double y, double L) {   // y >= L for y >= +0, L > 0
  return __double_as_longlong(y) >= __double_as_longlong(L);
}

// one thread per coordinate (coalesced over the flat [N][3] arrays)
__global__ void drift_kernel(int64_t n3, double *__restrict__ x, const double *__restrict__ v, double dt,
                             double L0, double L1, double L2, int p0, int p1, int p2) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n3) return;
  // the coordinate index without a 64-bit division (n3 < 2^32 for every
  // context that fits a GPU: 3 x 2^31 atoms would need 48 GB per array)
  const int k = n3 < (int64_t)0xffffffff ? (int)((uint32_t)j % 3u) : (int)(j % 3);
  const double L = k == 0 ? L0 : (k == 1 ? L1 : L2);
  const int per = k == 0 ? p0 : (k == 1 ? p1 : p2);
  // no contraction: x + v dt rounds the product and the sum separately
  double y = __dadd_rn(x[j], __dmul_rn(v[j], dt));
  if (per) {
    // one period at most per step; the same result as a floored modulo
    if (neg_bits(y) && y != 0.0) y += L;
    else if (ge_bits(y, L)) y -= L;
    if ((neg_bits(y) && y != 0.0) || (!neg_bits(y) && __double_as_longlong(y) > __double_as_longlong(L))) {
      y = fmod(y, L);
      if (y < 0.0) y += L;
    }
  }
  x[j] = y;
}

__global__ void philox_normals_kernel(const int64_t *__restrict__ ids, int64_t n, uint64_t step, uint64_t seed,
                                      double *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float g[3];
  gauss3((uint64_t)ids[i], step, seed, g);
  out[3 * i + 0] = g[0];
  out[3 * i + 1] = g[1];
  out[3 * i + 2] = g[2];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// scal[8] accumulates E_lat; scal[9] holds the stopped-atom counter (as u64 bits)
cudaError_t launch_couple(Ctx &c, double *v, double dt_md) {
  const double gdt = c.gammaL * dt_md;
  const double e1 = std::exp(-gdt);
  const double one_m_e2 = 1.0 - std::exp(-2.0 * gdt);
  const double kv = kKB * one_m_e2;
  const double kv0 = kv / (c.mt.m[0] * kMVV);
  if (c.n > 0)
    couple_kernel<<<nblk(c.n, 256), 256, 0, c.stream>>>(
        c.n, c.perm, c.type_s, c.mt, kv, kv0, c.Tl_d, c.A, c.T[c.tcur], v, c.dKE, c.p.couple_mode, c.p.frozen, c.p.seed,
        (uint64_t)c.md_step, e1,
        c.local ? kEVJ / (c.vatom * 1e-30 * c.p.gamma_Ce * c.p.Tmax_K * c.p.Tmax_K) : 1.0 / c.VC,
        reinterpret_cast<unsigned long long *>(c.scal + 9), c.local ? c.coef_host->thc : 0.0,
        c.local ? 1.0 / c.p.Tmax_K : 0.0,
        c.p.stop_beta_per_fs > 0 ? -std::expm1(-2.0 * c.p.stop_beta_per_fs * dt_md) : 0.0, c.p.stop_ecut_eV);
  sum_partial<<<kRedBlocks, kRedThreads, 0, c.stream>>>(c.n, c.dKE, c.partials);
  sum_final_accumulate<<<1, kRedThreads, 0, c.stream>>>(kRedBlocks, c.partials, c.scal + 8);
  return cudaGetLastError();
}

cudaError_t launch_drift(Ctx &c, double *x, const double *v, double dt) {
  if (c.n > 0)
    drift_kernel<<<nblk(3 * c.n, 256), 256, 0, c.stream>>>(3 * c.n, x, v, dt, c.box[0], c.box[1], c.box[2],
                                                               c.g.per[0], c.g.per[1], c.g.per[2]);
  return cudaGetLastError();
}

cudaError_t launch_philox_normals(const int64_t *ids, int64_t n, uint64_t step, uint64_t seed, double *out,
                                  cudaStream_t s) {
  if (n > 0) philox_normals_kernel<<<nblk(n, 256), 256, 0, s>>>(ids, n, step, seed, out);
  return cudaGetLastError();
}

}  // namespace ehc
