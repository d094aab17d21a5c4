// kernels_md.cu -- the lattice side of Eq. Motion: interatomic forces F_i from a
// shifted-force Morse pair potential on the neighbour list of the last build,
// the velocity-Verlet kick, and the largest speed (for a variable MD step).
//
//   phi(r)    = D [exp(-2 alpha (r - r0)) - 2 exp(-alpha (r - r0))]
//   phi_sf(r) = phi(r) - phi(r_c) - (r - r_c) phi'(r_c)      (zero energy and force at r_c)
//   F_i = sum_j phi_sf'(r_ij) (x_j - x_i) / r_ij,   E = (1/2) sum_i sum_j phi_sf(r_ij)
//
// Displacements are the exact integer minimum-image differences of the sorted
// quantised positions (2^-20 A grid); below 2^24 grid units (16 A) they convert
// to single precision exactly, so the pair geometry is exact before the first
// rounding.  Pair terms and the per-atom sums are single precision; the energy
// sum and the output forces are FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr int kMdThreads = 256;
constexpr double kMVVmd = 1.66053906660e-27 * 1.0e10 / 1.602176634e-19;  // amu (A/fs)^2 -> eV

struct MorseF {
  float D, alpha, r0, rc, pc, dpc;   // pc, dpc: phi(r_c), phi'(r_c)
  int32_t L[3], half[3];             // box on the grid and floor(L / 2) (0: axis not periodic)
};

// minimum image on the grid: both coordinates lie in [0, L) with L < 2^31, so the
// difference fits in int32; 2 d > L  <=>  d > floor(L / 2) for integers (a
// displacement of exactly half the box keeps its sign, as in the neighbour search)
__device__ __forceinline__ int32_t min_image(int32_t d, int32_t L, int32_t half) {
  if (half > 0) {
    if (d > half) d -= L;
    else if (d < -half) d += L;
  }
  return d;
}

__device__ __forceinline__ double blk_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  __syncthreads();
  return r;
}

// one thread per sorted atom; forces written in caller order (perm); block
// partial sums of the energy in part[blockIdx.x]
__global__ void __launch_bounds__(kMdThreads) morse_force_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt, const int4 *__restrict__ q_s,
    MorseF m, const int32_t *__restrict__ perm, double *__restrict__ F, double *__restrict__ part,
    int32_t *__restrict__ err) {
  __shared__ double sh[kMdThreads / 32];
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  float e = 0.0f;
  if (s < n) {
    const int4 qi = q_s[s];
    const int c = cnt[s];
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
    const float unit = 9.5367431640625e-07f;   // 2^-20 A
    for (int j = 0; j < c; ++j) {
      const int32_t t = checked_index(__ldg(nbr + (int64_t)j * n + s), n, err);
      const int4 qj = q_s[t];
      const float dx = (float)min_image(qj.x - qi.x, m.L[0], m.half[0]) * unit;
      const float dy = (float)min_image(qj.y - qi.y, m.L[1], m.half[1]) * unit;
      const float dz = (float)min_image(qj.z - qi.z, m.L[2], m.half[2]) * unit;
      const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
      const float e1 = expf(-m.alpha * (r - m.r0));
      const float phi = m.D * fmaf(e1, e1, -2.0f * e1);
      const float dphi = -2.0f * m.alpha * m.D * fmaf(e1, e1, -e1);
      const float phs = phi - m.pc - (r - m.rc) * m.dpc;
      const float w = (dphi - m.dpc) / r;
      fx = fmaf(w, dx, fx);
      fy = fmaf(w, dy, fy);
      fz = fmaf(w, dz, fz);
      e += 0.5f * phs;
    }
    const int64_t o = perm[s];
    F[3 * o + 0] = (double)fx;
    F[3 * o + 1] = (double)fy;
    F[3 * o + 2] = (double)fz;
  }
  const double r = blk_sum((double)e, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kMdThreads) md_sum_final(int nb, const double *__restrict__ part,
                                                           double *__restrict__ out) {
  __shared__ double sh[kMdThreads / 32];
  double a = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) a += part[k];
  const double r = blk_sum(a, sh);
  if (threadIdx.x == 0) *out = r;
}

// v_i += dt F_i / m_i (caller order)
__global__ void kick_kernel(int64_t n, double *__restrict__ v, const double *__restrict__ F,
                            const int32_t *__restrict__ type, MassTable mt, double dt_over_mvv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double c = dt_over_mvv / mt.m[type ? type[i] : 0];
  v[3 * i + 0] += c * F[3 * i + 0];
  v[3 * i + 1] += c * F[3 * i + 1];
  v[3 * i + 2] += c * F[3 * i + 2];
}

// block maxima of |v|^2 (caller order)
__global__ void __launch_bounds__(kMdThreads) vmax_partial(int64_t n, const double *__restrict__ v,
                                                           double *__restrict__ part) {
  __shared__ double sh[kMdThreads / 32];
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[3 * i], y = v[3 * i + 1], z = v[3 * i + 2];
    a = fmax(a, x * x + y * y + z * z);
  }
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kMdThreads / 32; ++w) r = fmax(r, sh[w]);
    part[blockIdx.x] = r;
  }
}

__global__ void vmax_final(int nb, const double *__restrict__ part, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double r = 0.0;
  for (int k = 0; k < nb; ++k) r = fmax(r, part[k]);
  *out = sqrt(r);
}

inline unsigned mblk(int64_t n) { return (unsigned)((n + kMdThreads - 1) / kMdThreads); }

}  // namespace

int md_force_blocks(int64_t n) { return (int)mblk(n > 0 ? n : 1); }

cudaError_t launch_forces(Ctx &c, double *F, double *part, double *out) {
  const int nb = md_force_blocks(c.n);
  if (c.n > 0) {
    double pc = 0.0, dpc = 0.0;
    {
      const double e1 = std::exp(-c.p.pot_alpha_perA * (c.p.rc_A - c.p.pot_r0_A));
      pc = c.p.pot_D_eV * (e1 * e1 - 2.0 * e1);
      dpc = -2.0 * c.p.pot_alpha_perA * c.p.pot_D_eV * (e1 * e1 - e1);
    }
    MorseF m{(float)c.p.pot_D_eV, (float)c.p.pot_alpha_perA, (float)c.p.pot_r0_A, (float)c.p.rc_A,
             (float)pc, (float)dpc, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < 3; ++k) {
      m.L[k] = (int32_t)c.g.Lq[k];
      m.half[k] = c.g.per[k] ? (int32_t)(c.g.Lq[k] / 2) : 0;
    }
    morse_force_kernel<<<nb, kMdThreads, 0, c.stream>>>((int32_t)c.n, c.nbr, c.cnt, c.q_s, m, c.perm, F, part,
                                                        c.err);
  }
  md_sum_final<<<1, kMdThreads, 0, c.stream>>>(c.n > 0 ? nb : 0, part, out);
  return cudaGetLastError();
}

cudaError_t launch_kick(Ctx &c, double *v, const double *F, double dt) {
  if (c.n > 0)
    kick_kernel<<<mblk(c.n), kMdThreads, 0, c.stream>>>(c.n, v, F, c.mt.n_types > 1 ? c.type_orig : nullptr, c.mt,
                                                        dt / kMVVmd);
  return cudaGetLastError();
}

cudaError_t launch_vmax(Ctx &c, const double *v, double *part, int nb, double *out) {
  if (c.n > 0) vmax_partial<<<nb, kMdThreads, 0, c.stream>>>(c.n, v, part);
  vmax_final<<<1, 32, 0, c.stream>>>(c.n > 0 ? nb : 0, part, out);
  return cudaGetLastError();
}

}  // namespace ehc
