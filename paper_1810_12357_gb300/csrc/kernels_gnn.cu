// kernels_gnn.cu -- the learned corrector network of the window propagator:
// forward (node features, tensor-core node MLP, edge MLP and pair flux),
// backward (edge MLP, tensor-core activation gradients, weight gradients) and
// the parameter update.
//
// The corrector adds a learned pair flux to the result Y of a propagator window
// (Eq. HeatTransport stands behind the window; the paper has no network):
//   delta_i = (Y_i - Tref) / Tmax,  D_ij = (delta_j - delta_i) / sigma,
//   q_ij = D^2 / (1 + D^2),  rho_ij = r_ij / r_c,  f_i = [Y_i / 1e4, T_l,i / 1e3, z_i / 18]
//   in_i = [f_i, <f_j>, <q>, <q^2>, <rho>, <q rho>, 1, 0 x 5]                (mean over the row)
//   h1 = relu(W1 in + b1),  h2 = relu(W2 h1 + b2),  u = W3 h2                (64, 64, 16)
//   z_ij = (u_i + u_j) + (P e_ij + b4),  g_ij = w4 . relu(z_ij)
//   Y^_i = Y_i + kappa Tmax sum_j (delta_j - delta_i) g_ij
// The node MLP runs on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32
// accumulation): one warp takes 16 nodes, the C fragments of a layer become
// the A fragments of the next in registers.  Weights and the stored
// activations (in, u) are BF16; the edge arithmetic is FP32.  Both atoms of a
// pair evaluate z_ij with the same operations on the same operands, so g_ij is
// bitwise symmetric, the pair terms (delta_j - delta_i) g_ij are exact
// negatives, and with compensated (TwoSum) row sums the correction keeps
// sum_i Y_i.
// Parameters (6336): [W1 (64 x 16) | b1 | W2 (64 x 64) | b2 | W3 (16 x 64) | P (16 x 2) | b4 | w4],
// matrices row-major (out x in).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

constexpr int kH = 64, kU = 16, kF = 16;
constexpr int oW1 = 0, ob1 = oW1 + kH * kF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              oP = oW3 + kU * kH, ob4 = oP + 2 * kU, ow4 = ob4 + kU, kNP = ow4 + kU;
static_assert(kNP == kGnnParams, "parameter count");
constexpr int kMlpThreads = 128;   // 4 warps x 16 nodes per slab
constexpr int kEdgeThreads = 128;
constexpr int kBwdTile = 64;       // nodes per backward tile (4 warps x 16)

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// D = A B + C, A 16 x 16 (row), B 16 x 8 (col), BF16 in, FP32 accumulate.  Fragment
// layout (g = lane / 4, t = lane % 4): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 =
// A[g][2t+8..], a3 = A[g+8][2t+8..]; b0 = B[2t..2t+1][g], b1 = B[2t+8..][g];
// c0,c1 = C[g][2t..2t+1], c2,c3 = C[g+8][2t..2t+1].
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// minimum image on the fixed-point grid: an exact half box is kept as is
__device__ __forceinline__ int64_t min_image(int64_t d, int64_t L, int per) {
  if (per) {
    if (2 * d > L) d -= L;
    else if (2 * d < -L) d += L;
  }
  return d;
}

struct GeoArgs {
  int64_t L0, L1, L2;
  int p0, p1, p2;
  float inv_rc;   // 1 / r_c [1/A]
};

__device__ __forceinline__ float pair_rho(int4 a, int4 b, const GeoArgs &g) {
  const int64_t dx = min_image((int64_t)b.x - a.x, g.L0, g.p0);
  const int64_t dy = min_image((int64_t)b.y - a.y, g.L1, g.p1);
  const int64_t dz = min_image((int64_t)b.z - a.z, g.L2, g.p2);
  const float r2 = (float)(dx * dx + dy * dy + dz * dz);
  return sqrtf(r2) * (9.5367431640625e-07f * g.inv_rc);   // 2^-20 A per grid unit
}

__device__ __forceinline__ float edge_q(float di, float dj, float inv_sigma) {
  const float D = (dj - di) * inv_sigma;
  const float D2 = D * D;
  return D2 / (1.0f + D2);
}

// layer-1 inputs of every atom (sorted order), BF16 [n][16]
__global__ void __launch_bounds__(256) gnn_feat_kernel(int32_t n, const int32_t *__restrict__ nbr,
                                                       const uint8_t *__restrict__ cnt, const int4 *__restrict__ q,
                                                       GeoArgs geo, const float *__restrict__ y,
                                                       const float *__restrict__ uTl, float Tref, float Tmax,
                                                       float inv_sigma, __nv_bfloat16 *__restrict__ in) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float di = y[s];
  const float ui = uTl[s];
  const int c = cnt[s];
  const int4 qi = q[s];
  float sf0 = 0.f, sf1 = 0.f, sf2 = 0.f, sq = 0.f, sq2 = 0.f, sr = 0.f, sqr = 0.f;
  for (int k = 0; k < c; ++k) {
    const int32_t t = nbr[(int64_t)k * n + s];
    const float dj = y[t];
    const float qq = edge_q(di, dj, inv_sigma);
    const float rho = pair_rho(qi, q[t], geo);
    const float uj = uTl[t];
    sf0 += fmaf(Tmax, dj, Tref) * 1.0e-4f;
    sf1 += (uj == uj) ? (Tref - uj) * 1.0e-3f : 0.0f;
    sf2 += (float)cnt[t] * (1.0f / 18.0f);
    sq += qq;
    sq2 += qq * qq;
    sr += rho;
    sqr += qq * rho;
  }
  const float inv = c > 0 ? 1.0f / (float)c : 0.0f;
  uint32_t w[8];
  w[0] = pack_bf16(fmaf(Tmax, di, Tref) * 1.0e-4f, (ui == ui) ? (Tref - ui) * 1.0e-3f : 0.0f);
  w[1] = pack_bf16((float)c * (1.0f / 18.0f), sf0 * inv);
  w[2] = pack_bf16(sf1 * inv, sf2 * inv);
  w[3] = pack_bf16(sq * inv, sq2 * inv);
  w[4] = pack_bf16(sr * inv, sqr * inv);
  w[5] = pack_bf16(1.0f, 0.0f);
  w[6] = 0u;
  w[7] = 0u;
  uint4 *dst = reinterpret_cast<uint4 *>(in + (int64_t)s * kF);
  dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
  dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// weights of the node MLP in shared memory: W1 [64][16], W2 [64][64], W3 [16][64]
// (row-major out x in, so that a B fragment's k pair is one 32-bit word), and for
// the backward the transposes W2T [64][64], W3T [64][16]
struct __align__(16) MlpSmem {
  __nv_bfloat16 W1[kH * kF], W2[kH * kH], W3[kU * kH];
  float b1[kH], b2[kH];
};
struct MlpSmemT {
  __nv_bfloat16 W2T[kH * kH], W3T[kH * kU];
};

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// B fragments of two n-tiles (nt, nt + 1) and one k-chunk of a weight matrix held
// row-major [N][K] in shared memory, by one ldmatrix.x4: lane l addresses row
// (nt + l / 16) * 8 + l % 8 at column kc * 16 + ((l / 8) % 2) * 8; the four 8 x 8
// matrices come back as b0, b1 of tile nt and b0, b1 of tile nt + 1
__device__ __forceinline__ void ldsm_b2(const __nv_bfloat16 *W, int K, int nt, int kc, int lane, uint32_t b[4]) {
  const __nv_bfloat16 *p = W + ((nt + (lane >> 4)) * 8 + (lane & 7)) * K + kc * 16 + ((lane >> 3) & 1) * 8;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
               : "r"(a));
}

// A fragment of a 16 x 16 slab of a row-major [n][16] BF16 array (rows past n are 0)
__device__ __forceinline__ void load_a16(const __nv_bfloat16 *__restrict__ x, int64_t row0, int32_t n, int g, int t,
                                         uint32_t a[4]) {
  const int64_t r0 = row0 + g, r1 = r0 + 8;
  a[0] = r0 < n ? ld32(x + r0 * 16 + 2 * t) : 0u;
  a[1] = r1 < n ? ld32(x + r1 * 16 + 2 * t) : 0u;
  a[2] = r0 < n ? ld32(x + r0 * 16 + 2 * t + 8) : 0u;
  a[3] = r1 < n ? ld32(x + r1 * 16 + 2 * t + 8) : 0u;
}

// C fragments [16 x 64] (8 n-tiles) + bias, relu -> A fragments (4 k-chunks); the
// pre-activations stay in c for the backward's masks
__device__ __forceinline__ void relu_to_a(const float c[8][4], const float *bias, int t, uint32_t a[4][4]) {
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    const int c0 = 16 * kc + 2 * t, c1 = c0 + 8;
    const float *x = c[2 * kc], *y = c[2 * kc + 1];
    a[kc][0] = pack_bf16(fmaxf(x[0] + bias[c0], 0.f), fmaxf(x[1] + bias[c0 + 1], 0.f));
    a[kc][1] = pack_bf16(fmaxf(x[2] + bias[c0], 0.f), fmaxf(x[3] + bias[c0 + 1], 0.f));
    a[kc][2] = pack_bf16(fmaxf(y[0] + bias[c1], 0.f), fmaxf(y[1] + bias[c1 + 1], 0.f));
    a[kc][3] = pack_bf16(fmaxf(y[2] + bias[c1], 0.f), fmaxf(y[3] + bias[c1 + 1], 0.f));
  }
}

// forward of one 16-node slab: c1 = in W1^T (pre-bias), h1 = relu(c1 + b1),
// c2 = h1 W2^T, h2 = relu(c2 + b2), c3 = h2 W3^T
__device__ __forceinline__ void mlp_slab(const MlpSmem &w, const uint32_t ain[4], int g, int t, float c1[8][4],
                                         uint32_t h1[4][4], float c2[8][4], uint32_t h2[4][4], float c3[2][4]) {
  const int lane = threadIdx.x & 31;
  uint32_t b[4];
#pragma unroll
  for (int nt = 0; nt < 8; nt += 2) {
    c1[nt][0] = c1[nt][1] = c1[nt][2] = c1[nt][3] = 0.f;
    c1[nt + 1][0] = c1[nt + 1][1] = c1[nt + 1][2] = c1[nt + 1][3] = 0.f;
    ldsm_b2(w.W1, kF, nt, 0, lane, b);
    mma16816(c1[nt], ain, b[0], b[1]);
    mma16816(c1[nt + 1], ain, b[2], b[3]);
  }
  relu_to_a(c1, w.b1, t, h1);
#pragma unroll
  for (int nt = 0; nt < 8; nt += 2) {
    c2[nt][0] = c2[nt][1] = c2[nt][2] = c2[nt][3] = 0.f;
    c2[nt + 1][0] = c2[nt + 1][1] = c2[nt + 1][2] = c2[nt + 1][3] = 0.f;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      ldsm_b2(w.W2, kH, nt, kc, lane, b);
      mma16816(c2[nt], h1[kc], b[0], b[1]);
      mma16816(c2[nt + 1], h1[kc], b[2], b[3]);
    }
  }
  relu_to_a(c2, w.b2, t, h2);
  c3[0][0] = c3[0][1] = c3[0][2] = c3[0][3] = 0.f;
  c3[1][0] = c3[1][1] = c3[1][2] = c3[1][3] = 0.f;
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    ldsm_b2(w.W3, kH, 0, kc, lane, b);
    mma16816(c3[0], h2[kc], b[0], b[1]);
    mma16816(c3[1], h2[kc], b[2], b[3]);
  }
  (void)g;
}

__device__ __forceinline__ void load_mlp_weights(const __nv_bfloat16 *__restrict__ wb, MlpSmem &w) {
  for (int k = threadIdx.x; k < kH * kF; k += blockDim.x) w.W1[k] = wb[oW1 + k];
  for (int k = threadIdx.x; k < kH * kH; k += blockDim.x) w.W2[k] = wb[oW2 + k];
  for (int k = threadIdx.x; k < kU * kH; k += blockDim.x) w.W3[k] = wb[oW3 + k];
  for (int k = threadIdx.x; k < kH; k += blockDim.x) {
    w.b1[k] = __bfloat162float(wb[ob1 + k]);
    w.b2[k] = __bfloat162float(wb[ob2 + k]);
  }
}

// node MLP: u [n][16] BF16 from the layer-1 inputs; grid-stride over 16-node slabs
__global__ void __launch_bounds__(kMlpThreads, 8) gnn_mlp_kernel(int32_t n, const __nv_bfloat16 *__restrict__ in,
                                                              const __nv_bfloat16 *__restrict__ wb,
                                                              __nv_bfloat16 *__restrict__ u) {
  __shared__ MlpSmem w;
  load_mlp_weights(wb, w);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t nslab = ((int64_t)n + 15) / 16;
  for (int64_t sl = (int64_t)blockIdx.x * (kMlpThreads / 32) + warp; sl < nslab;
       sl += (int64_t)gridDim.x * (kMlpThreads / 32)) {
    const int64_t row0 = sl * 16;
    uint32_t ain[4];
    load_a16(in, row0, n, g, t, ain);
    float c1[8][4], c2[8][4], c3[2][4];
    uint32_t h1[4][4], h2[4][4];
    mlp_slab(w, ain, g, t, c1, h1, c2, h2, c3);
    const int64_t r0 = row0 + g, r1 = r0 + 8;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int col = nt * 8 + 2 * t;
      if (r0 < n) *reinterpret_cast<uint32_t *>(u + r0 * kU + col) = pack_bf16(c3[nt][0], c3[nt][1]);
      if (r1 < n) *reinterpret_cast<uint32_t *>(u + r1 * kU + col) = pack_bf16(c3[nt][2], c3[nt][3]);
    }
  }
}

// the edge layer's weights as FP32 (from their BF16 values)
struct EdgeW {
  float P0[kU], P1[kU], b4[kU], w4[kU];
};

__device__ __forceinline__ void load_edge_w(const __nv_bfloat16 *__restrict__ wb, EdgeW &e) {
  for (int k = threadIdx.x; k < kU; k += blockDim.x) {
    e.P0[k] = __bfloat162float(wb[oP + 2 * k]);
    e.P1[k] = __bfloat162float(wb[oP + 2 * k + 1]);
    e.b4[k] = __bfloat162float(wb[ob4 + k]);
    e.w4[k] = __bfloat162float(wb[ow4 + k]);
  }
}

__device__ __forceinline__ void load_u(const __nv_bfloat16 *__restrict__ u, int64_t s, float v[kU]) {
  const uint4 *p = reinterpret_cast<const uint4 *>(u + s * kU);
  const uint4 a = p[0], b = p[1];
  const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w[k]);
    v[2 * k] = __low2float(h);
    v[2 * k + 1] = __high2float(h);
  }
}

__device__ __forceinline__ void two_sum_acc(float &F, float &Fc, float x) {
  const float s = __fadd_rn(F, x);
  const float bb = __fsub_rn(s, F);
  const float e = __fadd_rn(__fsub_rn(F, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  Fc = __fadd_rn(Fc, e);
  F = s;
}

// g_ij from both atoms' node states and the pair's symmetric edge features: the
// same operations in the same order on either side
__device__ __forceinline__ float pair_g(const float ui[kU], const float uj[kU], float qq, float rho, const EdgeW &e,
                                        float zr[kU]) {
  float gsum = 0.f;
#pragma unroll
  for (int k = 0; k < kU; ++k) {
    const float z = __fadd_rn(ui[k], uj[k]) + fmaf(e.P0[k], qq, fmaf(e.P1[k], rho, e.b4[k]));
    zr[k] = z;
    gsum = fmaf(e.w4[k], fmaxf(z, 0.f), gsum);
  }
  return gsum;
}

// Y^ = Y + kappa Tmax sum_j (delta_j - delta_i) g_ij on the sorted state: T (FP64)
// in place and the mirror y (delta) with it; dY (optional) the correction [K]
__global__ void __launch_bounds__(kEdgeThreads) gnn_edge_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt, const int4 *__restrict__ q,
    GeoArgs geo, const float *__restrict__ y, const __nv_bfloat16 *__restrict__ u, const __nv_bfloat16 *__restrict__ wb,
    float inv_sigma, double kT, double invTmax, double *__restrict__ T, float *__restrict__ y_out,
    double *__restrict__ dY) {
  __shared__ EdgeW e;
  load_edge_w(wb, e);
  __syncthreads();
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float di = y[s];
  const int c = cnt[s];
  const int4 qi = q[s];
  float ui[kU], uj[kU], zr[kU];
  load_u(u, s, ui);
  float F = 0.f, Fc = 0.f;
  for (int k = 0; k < c; ++k) {
    const int32_t t = nbr[(int64_t)k * n + s];
    const float dj = y[t];
    load_u(u, t, uj);
    const float gij = pair_g(ui, uj, edge_q(di, dj, inv_sigma), pair_rho(qi, q[t], geo), e, zr);
    two_sum_acc(F, Fc, __fmul_rn(dj - di, gij));
  }
  const double d = kT * ((double)F + (double)Fc);
  if (dY) dY[s] = d;
  T[s] += d;
  y_out[s] = di + (float)(d * invTmax);
}

// ---- backward ----

// dL/dY^_i of the window loss L = (1/N) sum ((Y^ - T*)/T*)^2, and the loss's block sums
__global__ void __launch_bounds__(256) gnn_loss_kernel(int32_t n, const double *__restrict__ Yh,
                                                       const double *__restrict__ Ts, double inv_n,
                                                       float *__restrict__ G, double *__restrict__ lpart) {
  __shared__ double red[8];
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (s < n) {
    const double r = (Yh[s] - Ts[s]) / Ts[s];
    l = r * r;
    G[s] = (float)(2.0 * r * inv_n / Ts[s]);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < 8; ++w) a += red[w];
    lpart[blockIdx.x] = a * inv_n;
  }
}

// edge layer backward, one thread per atom m (its own directed edges for the edge
// weights; both directions of each pair for du_m):
//   dg_mj = kappa Tmax (delta_j - delta_m) G_m
//   dw4 += dg relu(z),  dz = dg w4 [z > 0],  dP += dz (q, rho),  db4 += dz
//   du_m = sum_j kappa Tmax (delta_j - delta_m)(G_m - G_j) w4 [z_mj > 0]
// du [n][16] FP32; the edge weights' block sums into epart [block][64]
__global__ void __launch_bounds__(kEdgeThreads) gnn_edge_bwd_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt, const int4 *__restrict__ q,
    GeoArgs geo, const float *__restrict__ y, const __nv_bfloat16 *__restrict__ u, const __nv_bfloat16 *__restrict__ wb,
    float inv_sigma, float kT, const float *__restrict__ G, float *__restrict__ du, float *__restrict__ epart) {
  __shared__ EdgeW e;
  __shared__ float red[kEdgeThreads / 32][4 * kU];
  load_edge_w(wb, e);
  __syncthreads();
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  float aw4[kU], aP0[kU], aP1[kU], ab4[kU], dum[kU];
#pragma unroll
  for (int k = 0; k < kU; ++k) aw4[k] = aP0[k] = aP1[k] = ab4[k] = dum[k] = 0.f;
  if (s < n) {
    const float di = y[s];
    const float gm = G[s];
    const int c = cnt[s];
    const int4 qi = q[s];
    float ui[kU], uj[kU], zr[kU];
    load_u(u, s, ui);
    for (int k = 0; k < c; ++k) {
      const int32_t t = nbr[(int64_t)k * n + s];
      const float dj = y[t];
      load_u(u, t, uj);
      const float qq = edge_q(di, dj, inv_sigma);
      const float rho = pair_rho(qi, q[t], geo);
      pair_g(ui, uj, qq, rho, e, zr);
      const float dYk = kT * (dj - di);
      const float dg = dYk * gm;
      const float dgu = dYk * (gm - G[t]);
#pragma unroll
      for (int m = 0; m < kU; ++m) {
        const bool on = zr[m] > 0.f;
        aw4[m] = fmaf(dg, on ? zr[m] : 0.f, aw4[m]);
        const float dz = on ? dg * e.w4[m] : 0.f;
        aP0[m] = fmaf(dz, qq, aP0[m]);
        aP1[m] = fmaf(dz, rho, aP1[m]);
        ab4[m] += dz;
        dum[m] = fmaf(on ? dgu : 0.f, e.w4[m], dum[m]);
      }
    }
    float4 *dst = reinterpret_cast<float4 *>(du + (int64_t)s * kU);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = make_float4(dum[4 * k], dum[4 * k + 1], dum[4 * k + 2], dum[4 * k + 3]);
  }
  // block sums of the edge weights' gradients: [P0 P1 interleaved as P (16 x 2) | b4 | w4]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < kU; ++m) {
    float v0 = aP0[m], v1 = aP1[m], v2 = ab4[m], v3 = aw4[m];
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_down_sync(0xffffffffu, v0, o);
      v1 += __shfl_down_sync(0xffffffffu, v1, o);
      v2 += __shfl_down_sync(0xffffffffu, v2, o);
      v3 += __shfl_down_sync(0xffffffffu, v3, o);
    }
    if (lane == 0) {
      red[warp][2 * m] = v0;
      red[warp][2 * m + 1] = v1;
      red[warp][2 * kU + m] = v2;
      red[warp][3 * kU + m] = v3;
    }
  }
  __syncthreads();
  if (threadIdx.x < 4 * kU) {
    float a = 0.f;
    for (int w = 0; w < kEdgeThreads / 32; ++w) a += red[w][threadIdx.x];
    epart[(int64_t)blockIdx.x * 4 * kU + threadIdx.x] = a;
  }
}

// node MLP backward over tiles of 64 nodes (4 warps x 16): each warp recomputes its
// slab's forward on the tensor cores, then da2 = (du W3) [a2 > 0] and
// da1 = (da2 W2) [a1 > 0] (tensor cores, transposed weights), and stages in, h1,
// h2, da1, da2, du of the tile in shared memory (FP32); the weight gradients are
// then summed over the tile's nodes in FP32 by all threads (each thread owns
// fixed entries: the sums run in a fixed order, so results are reproducible).
// mpart [block][W1 | b1 | W2 | b2 | W3] block sums.
struct BwdStage {
  float in[kBwdTile][kF], h1[kBwdTile][kH], h2[kBwdTile][kH], da1[kBwdTile][kH], da2[kBwdTile][kH],
      du[kBwdTile][kU];
};
constexpr int kMlpPart = oP;   // W1, b1, W2, b2, W3 entries of a block's partial sums

__global__ void __launch_bounds__(kMlpThreads) gnn_mlp_bwd_kernel(int32_t n, const __nv_bfloat16 *__restrict__ in,
                                                                  const float *__restrict__ du,
                                                                  const __nv_bfloat16 *__restrict__ wb,
                                                                  float *__restrict__ mpart) {
  __shared__ MlpSmem w;
  __shared__ MlpSmemT wt;
  extern __shared__ __align__(16) float dyn[];
  BwdStage &st = *reinterpret_cast<BwdStage *>(dyn);
  load_mlp_weights(wb, w);
  for (int k = threadIdx.x; k < kH * kH; k += blockDim.x) {
    const int a = k / kH, b = k % kH;
    wt.W2T[b * kH + a] = wb[oW2 + k];   // W2T[in][out]
  }
  for (int k = threadIdx.x; k < kU * kH; k += blockDim.x) {
    const int a = k / kH, b = k % kH;   // W3[a][b], a < 16
    wt.W3T[b * kU + a] = wb[oW3 + k];
  }
  __syncthreads();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  // owned weight-gradient entries
  float aW2[32], aW1[8], aW3[8], ab = 0.f;
#pragma unroll
  for (int k = 0; k < 32; ++k) aW2[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) aW1[k] = aW3[k] = 0.f;
  const int64_t ntile = ((int64_t)n + kBwdTile - 1) / kBwdTile;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t row0 = tile * kBwdTile + warp * 16;
    uint32_t ain[4];
    load_a16(in, row0, n, g, t, ain);
    float c1[8][4], c2[8][4], c3[2][4];
    uint32_t h1[4][4], h2[4][4];
    mlp_slab(w, ain, g, t, c1, h1, c2, h2, c3);
    // du as an A fragment (K = 16)
    const int64_t r0 = row0 + g, r1 = r0 + 8;
    uint32_t adu[4];
    {
      const float *p0 = du + r0 * kU + 2 * t, *p1 = du + r1 * kU + 2 * t;
      adu[0] = r0 < n ? pack_bf16(p0[0], p0[1]) : 0u;
      adu[1] = r1 < n ? pack_bf16(p1[0], p1[1]) : 0u;
      adu[2] = r0 < n ? pack_bf16(p0[8], p0[9]) : 0u;
      adu[3] = r1 < n ? pack_bf16(p1[8], p1[9]) : 0u;
    }
    // da2 = (du W3) [a2 > 0]; B(k = u, n = h) = W3[u][h] = W3T[h][u]
    float d2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      d2[nt][0] = d2[nt][1] = d2[nt][2] = d2[nt][3] = 0.f;
      const __nv_bfloat16 *wr = wt.W3T + (nt * 8 + g) * kU + 2 * t;
      mma16816(d2[nt], adu, ld32(wr), ld32(wr + 8));
      const int col = nt * 8 + 2 * t;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (!(c2[nt][e] + w.b2[col + (e & 1)] > 0.f)) d2[nt][e] = 0.f;
    }
    uint32_t ad2[4][4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      ad2[kc][0] = pack_bf16(d2[2 * kc][0], d2[2 * kc][1]);
      ad2[kc][1] = pack_bf16(d2[2 * kc][2], d2[2 * kc][3]);
      ad2[kc][2] = pack_bf16(d2[2 * kc + 1][0], d2[2 * kc + 1][1]);
      ad2[kc][3] = pack_bf16(d2[2 * kc + 1][2], d2[2 * kc + 1][3]);
    }
    // da1 = (da2 W2) [a1 > 0]; B(k = out, n = in) = W2[k][n] = W2T[n][k]
    float d1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      d1[nt][0] = d1[nt][1] = d1[nt][2] = d1[nt][3] = 0.f;
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        const __nv_bfloat16 *wr = wt.W2T + (nt * 8 + g) * kH + 16 * kc + 2 * t;
        mma16816(d1[nt], ad2[kc], ld32(wr), ld32(wr + 8));
      }
      const int col = nt * 8 + 2 * t;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (!(c1[nt][e] + w.b1[col + (e & 1)] > 0.f)) d1[nt][e] = 0.f;
    }
    // stage this warp's 16 nodes (rows past n: zeros, so they add nothing)
    __syncthreads();   // the previous tile's sums are done with the staging area
    const int l0 = warp * 16 + g, l1 = l0 + 8;
    const bool v0 = r0 < n, v1 = r1 < n;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = nt * 8 + 2 * t;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float b1v = w.b1[col + e], b2v = w.b2[col + e];
        st.h1[l0][col + e] = v0 ? fmaxf(c1[nt][e] + b1v, 0.f) : 0.f;
        st.h1[l1][col + e] = v1 ? fmaxf(c1[nt][2 + e] + b1v, 0.f) : 0.f;
        st.h2[l0][col + e] = v0 ? fmaxf(c2[nt][e] + b2v, 0.f) : 0.f;
        st.h2[l1][col + e] = v1 ? fmaxf(c2[nt][2 + e] + b2v, 0.f) : 0.f;
        st.da1[l0][col + e] = v0 ? d1[nt][e] : 0.f;
        st.da1[l1][col + e] = v1 ? d1[nt][2 + e] : 0.f;
        st.da2[l0][col + e] = v0 ? d2[nt][e] : 0.f;
        st.da2[l1][col + e] = v1 ? d2[nt][2 + e] : 0.f;
      }
    }
    for (int k = lane; k < 16 * kF; k += 32) {
      const int r = k / kF, f = k % kF;
      const int64_t row = row0 + r;
      st.in[warp * 16 + r][f] = row < n ? __bfloat162float(in[row * kF + f]) : 0.f;
      st.du[warp * 16 + r][f] = row < n ? du[row * kU + f] : 0.f;
    }
    __syncthreads();
    // weight-gradient sums over the tile's nodes, in node order
    {
      const int b = tid & 63, a0 = tid >> 6;            // dW2[a][b], a = a0 + 2 k
      const int f = tid & 15, a1 = tid >> 4;            // dW1[a][f], a = a1 + 8 k
      const int hh = tid & 63, u0 = tid >> 6;           // dW3[u][hh], u = u0 + 2 k
      for (int r = 0; r < kBwdTile; ++r) {
        const float hb = st.h1[r][b];
#pragma unroll
        for (int k = 0; k < 32; ++k) aW2[k] = fmaf(st.da2[r][a0 + 2 * k], hb, aW2[k]);
        const float xf = st.in[r][f];
#pragma unroll
        for (int k = 0; k < 8; ++k) aW1[k] = fmaf(st.da1[r][a1 + 8 * k], xf, aW1[k]);
        const float h2v = st.h2[r][hh];
#pragma unroll
        for (int k = 0; k < 8; ++k) aW3[k] = fmaf(st.du[r][u0 + 2 * k], h2v, aW3[k]);
        ab += tid < kH ? st.da1[r][tid] : st.da2[r][tid - kH];
      }
    }
  }
  float *out = mpart + (int64_t)blockIdx.x * kMlpPart;
  {
    const int b = tid & 63, a0 = tid >> 6;
#pragma unroll
    for (int k = 0; k < 32; ++k) out[oW2 + (a0 + 2 * k) * kH + b] = aW2[k];
    const int f = tid & 15, a1 = tid >> 4;
#pragma unroll
    for (int k = 0; k < 8; ++k) out[oW1 + (a1 + 8 * k) * kF + f] = aW1[k];
    const int hh = tid & 63, u0 = tid >> 6;
#pragma unroll
    for (int k = 0; k < 8; ++k) out[oW3 + (u0 + 2 * k) * kH + hh] = aW3[k];
    if (tid < kH) out[ob1 + tid] = ab;
    else out[ob2 + tid - kH] = ab;
  }
}

// gradient = sums of the blocks' partials (fixed order), one thread per parameter
__global__ void gnn_grad_reduce_kernel(int nb_m, const float *__restrict__ mpart, int nb_e,
                                       const float *__restrict__ epart, float *__restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kNP) return;
  float a = 0.f;
  if (k < kMlpPart) {
    for (int b = 0; b < nb_m; ++b) a += mpart[(int64_t)b * kMlpPart + k];
  } else {
    const int j = k - kMlpPart;   // P (32) | b4 (16) | w4 (16): the edge partials' layout
    for (int b = 0; b < nb_e; ++b) a += epart[(int64_t)b * 4 * kU + j];
  }
  grad[k] = a;
}

// Adam on the FP32 master weights, then their BF16 copy
__global__ void gnn_adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                                const float *__restrict__ gr, float lr, float b1t, float b2t,
                                __nv_bfloat16 *__restrict__ pb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kNP) return;
  const float g = gr[k];
  const float mk = 0.9f * m[k] + 0.1f * g;
  const float vk = 0.999f * v[k] + 0.001f * g * g;
  m[k] = mk;
  v[k] = vk;
  const float mh = mk / (1.0f - b1t), vh = vk / (1.0f - b2t);
  const float pk = p[k] - lr * mh / (sqrtf(vh) + 1e-8f);
  p[k] = pk;
  pb[k] = __float2bfloat16_rn(pk);
}

__global__ void gnn_to_bf16_kernel(const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kNP) pb[k] = __float2bfloat16_rn(p[k]);
}

__global__ void gnn_sum_kernel(int nb, const double *__restrict__ part, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0;
  for (int b = 0; b < nb; ++b) a += part[b];
  *out = a;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

GeoArgs geo_of(const Ctx &c) {
  GeoArgs g;
  g.L0 = c.g.Lq[0];
  g.L1 = c.g.Lq[1];
  g.L2 = c.g.Lq[2];
  g.p0 = c.g.per[0];
  g.p1 = c.g.per[1];
  g.p2 = c.g.per[2];
  g.inv_rc = (float)(1.0 / c.p.rc_A);
  return g;
}

}  // namespace

// resident blocks: 8 per SM for the forward (64 registers, 128 threads), whose
// MMA chains need the warps to hide their latency
int gnn_mlp_blocks(Ctx &c) { return 8 * (c.num_sms > 0 ? c.num_sms : 152); }
int gnn_edge_blocks(int64_t n) { return (int)nblk(n > 0 ? n : 1, kEdgeThreads); }
int gnn_loss_blocks(int64_t n) { return (int)nblk(n > 0 ? n : 1, 256); }
size_t gnn_bwd_smem() { return sizeof(BwdStage); }

cudaError_t gnn_forward(Ctx &c, const __nv_bfloat16 *wb, double sigma, double kappa, const float *y,
                        __nv_bfloat16 *in, __nv_bfloat16 *u, double *T, float *y_out, double *dY) {
  if (c.n == 0) return cudaSuccess;
  const int32_t n = (int32_t)c.n;
  const GeoArgs geo = geo_of(c);
  const float Tref = (float)c.p.Tref_K, Tmax = (float)c.p.Tmax_K, isg = (float)(1.0 / sigma);
  gnn_feat_kernel<<<nblk(n, 256), 256, 0, c.stream>>>(n, c.nbr, c.cnt, c.q_s, geo, y, c.uTl, Tref, Tmax, isg, in);
  gnn_mlp_kernel<<<gnn_mlp_blocks(c), kMlpThreads, 0, c.stream>>>(n, in, wb, u);
  gnn_edge_kernel<<<nblk(n, kEdgeThreads), kEdgeThreads, 0, c.stream>>>(
      n, c.nbr, c.cnt, c.q_s, geo, y, u, wb, isg, kappa * c.p.Tmax_K, 1.0 / c.p.Tmax_K, T, y_out, dY);
  return cudaGetLastError();
}

cudaError_t gnn_backward(Ctx &c, const __nv_bfloat16 *wb, double sigma, double kappa, const float *y,
                         const __nv_bfloat16 *in, const __nv_bfloat16 *u, const double *Yh, const double *Ts,
                         float *G, float *du, double *lpart, double *loss, float *mpart, float *epart, float *grad) {
  if (c.n == 0) return cudaSuccess;
  const int32_t n = (int32_t)c.n;
  const GeoArgs geo = geo_of(c);
  const int nbl = gnn_loss_blocks(n);
  gnn_loss_kernel<<<nbl, 256, 0, c.stream>>>(n, Yh, Ts, 1.0 / (double)n, G, lpart);
  gnn_sum_kernel<<<1, 32, 0, c.stream>>>(nbl, lpart, loss);
  const int nbe = gnn_edge_blocks(n);
  gnn_edge_bwd_kernel<<<nbe, kEdgeThreads, 0, c.stream>>>(n, c.nbr, c.cnt, c.q_s, geo, y, u, wb,
                                                          (float)(1.0 / sigma), (float)(kappa * c.p.Tmax_K), G, du,
                                                          epart);
  const int nbm = gnn_mlp_blocks(c);
  gnn_mlp_bwd_kernel<<<nbm, kMlpThreads, sizeof(BwdStage), c.stream>>>(n, in, du, wb, mpart);
  gnn_grad_reduce_kernel<<<nblk(kNP, 256), 256, 0, c.stream>>>(nbm, mpart, nbe, epart, grad);
  return cudaGetLastError();
}

cudaError_t gnn_adam(cudaStream_t st, float *p, float *m, float *v, const float *g, float lr, int t,
                     __nv_bfloat16 *pb) {
  const float b1t = powf(0.9f, (float)t), b2t = powf(0.999f, (float)t);
  gnn_adam_kernel<<<nblk(kNP, 256), 256, 0, st>>>(p, m, v, g, lr, b1t, b2t, pb);
  return cudaGetLastError();
}

cudaError_t gnn_params_to_bf16(cudaStream_t st, const float *p, __nv_bfloat16 *pb) {
  gnn_to_bf16_kernel<<<nblk(kNP, 256), 256, 0, st>>>(p, pb);
  return cudaGetLastError();
}

cudaError_t gnn_setup(size_t smem) {
  return cudaFuncSetAttribute(gnn_mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace ehc
