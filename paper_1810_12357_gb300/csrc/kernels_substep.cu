// kernels_substep.cu -- the per-substep sweep of Eq. HeatTransport.
//
// For every atom i:
//   F_i  = sum_j f(theta_i, theta_j),
//   f(a, b) = b (1 - a) e^{a - b} - a (1 - b) e^{b - a}        (Delta e_ij = -(theta_i - theta_j))
//   T_i += dt [ Tmax K F_i - chi_i (G / C_e)(T_i - T_l,i) + q_i(t) ]
//   A_i += dt chi_i G V_atom (T_i - T_l,i)                    (Eq. RateExchange)
// All atoms read the previous substep's snapshot (Jacobi) through a
// double-buffered mirror.
//
// Single-precision path (flux_prec = 0).
//  * State: delta = (T - Tref) / Tmax held as an unevaluated float pair hi + lo
//    (about 48 significant bits); hi doubles as the mirror the neighbours read.
//    T is rebuilt in FP64 after every substep call (merge) and split again before
//    the next one.  The per-atom exchanged energy A_i is FP64.
//  * Pair term: with a = theta_i, b = theta_j, Delta = b - a and the symmetric
//    P = a + b - 2 a b (so that 2 a (1 - b) = P - Delta and b (1 - a) = a (1 - b) + Delta),
//        f(a, b) = b(1-a) e^{-Delta} - a(1-b) e^{Delta} = Delta cosh(Delta) - P sinh(Delta)
//                = Delta * B,   B = cosh(Delta) - P sinh(Delta)/Delta.
//    B depends on the pair only through Delta^2 and P, which both atoms compute
//    bit for bit alike (fl(a+b) = fl(b+a), and fma(-2a, b, s) = fma(-2b, a, s)),
//    so the two contributions are exactly +-Delta*B: pair fluxes cancel exactly
//    before each atom's own accumulation rounding.  B >= e^{-1} on [0,1]^2, so the
//    FP32 error is relative to the local temperature difference Delta.
//    cosh and sinh(Delta)/Delta come from their Taylor series in Delta^2, with
//    the order set per tile from the largest value spread of its rows (previous
//    substep): spread < 1.2e-4 -> B = 1 - P; < 0.02 -> to Delta^2; < 0.12 -> to
//    Delta^4; otherwise to Delta^10 (|Delta| <= 1).  Truncation stays below 3e-8
//    of B in every tier.  Two atoms whose rows use different tiers differ in B
//    by at most that bound; within a tier B is bit-identical on both sides.
//  * Row tiles: a CTA takes one row of cells at a time; the rows around it (at
//    most 9) are copied into shared memory by bulk copies (one producer warp,
//    mbarrier completion, two buffers) and neighbours are 16-bit indices into
//    that tile.
//
// Double-precision path (flux_prec = 1): gathers T itself and evaluates the pair
// term as written in the paper with one exponential, E = e^{theta_lo - theta_hi}:
// f(theta_lo, theta_hi) = theta_hi (1 - theta_lo) E - theta_lo (1 - theta_hi) / E.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "ehc_internal.cuh"

namespace ehc {

namespace {

// F += f(theta_i, theta_j) = Delta * B (see above).  ai = theta_i, m2ai = -2 theta_i.
template <int TIER>
__device__ __forceinline__ float pair_acc(float F, float di, float dj, float th, float ai, float m2ai) {
  const float D = dj - di;
  if (TIER == 3) {                                                  // B = 1 - P
    const float b = th + dj;
    const float P = fmaf(m2ai, b, ai + b);
    return fmaf(D, 1.0f - P, F);
  }
  const float x = D * D;
  float S, C;
  if (TIER == 2) {
    S = fmaf(x, 1.6666667e-01f, 1.0f);                              // 1 + D^2/3!
    C = fmaf(x, 0.5f, 1.0f);                                        // 1 + D^2/2!
  } else if (TIER == 1) {
    S = fmaf(x, fmaf(x, 8.3333333e-03f, 1.6666667e-01f), 1.0f);     // ... + D^4/5!
    C = fmaf(x, fmaf(x, 4.1666667e-02f, 0.5f), 1.0f);               // ... + D^4/4!
  } else {
    S = fmaf(x, 2.5052108e-08f, 2.7557319e-06f);                    // 1/11!, 1/9!
    S = fmaf(x, S, 1.9841270e-04f);                                 // 1/7!
    S = fmaf(x, S, 8.3333333e-03f);                                 // 1/5!
    S = fmaf(x, S, 1.6666667e-01f);                                 // 1/3!
    S = fmaf(x, S, 1.0f);
    C = fmaf(x, 2.7557319e-07f, 2.4801587e-05f);                    // 1/10!, 1/8!
    C = fmaf(x, C, 1.3888889e-03f);                                 // 1/6!
    C = fmaf(x, C, 4.1666667e-02f);                                 // 1/4!
    C = fmaf(x, C, 0.5f);
    C = fmaf(x, C, 1.0f);
  }
  const float b = th + dj;
  const float P = fmaf(m2ai, b, ai + b);
  return fmaf(D, fmaf(-P, S, C), F);
}

// the pair term alone, for the compensated sums: as pair_acc(0, ...), except
// that B = 1 - P is applied as one fused operation, Delta - Delta P with a single
// rounding (still exactly the negative of the partner's term: Delta changes
// sign, P does not, and round-to-nearest is odd)
template <int TIER>
__device__ __forceinline__ float pair_flux(float di, float dj, float th, float ai, float m2ai) {
  if (TIER == 3) {
    const float D = dj - di;
    const float b = th + dj;
    const float P = fmaf(m2ai, b, ai + b);
    return fmaf(-D, P, D);
  }
  return pair_acc<TIER>(0.0f, di, dj, th, ai, m2ai);
}

// fl(f(theta_i, theta_j)) = fl(Delta B) with the series order chosen from this
// pair's own Delta^2 (the same thresholds and truncation bounds as the row tiles'
// per-tile tiers): both atoms of a pair compute Delta^2 and P bit for bit alike,
// so they take the same branch and their terms are exact negatives.
__device__ __forceinline__ float pair_term(float di, float dj, float th, float ai, float m2ai) {
  const float D = dj - di;
  const float x = D * D;
  const float b = th + dj;
  const float P = fmaf(m2ai, b, ai + b);
  float B;
  if (x < 1.44e-8f) {                                             // |Delta| < 1.2e-4
    return fmaf(-D, P, D);                                        // Delta (1 - P), one rounding
  } else if (x < 4.0e-4f) {                                       // |Delta| < 0.02
    B = fmaf(-P, fmaf(x, 1.6666667e-01f, 1.0f), fmaf(x, 0.5f, 1.0f));
  } else if (x < 1.44e-2f) {                                      // |Delta| < 0.12
    B = fmaf(-P, fmaf(x, fmaf(x, 8.3333333e-03f, 1.6666667e-01f), 1.0f),
             fmaf(x, fmaf(x, 4.1666667e-02f, 0.5f), 1.0f));
  } else {
    return pair_acc<0>(0.0f, di, dj, th, ai, m2ai);
  }
  return __fmul_rn(D, B);
}

// (F, Fc) += t: TwoSum of F and t, the rounding error accumulated in Fc
__device__ __forceinline__ void two_sum_acc(float &F, float &Fc, float t) {
  const float s = __fadd_rn(F, t);
  const float bb = __fsub_rn(s, F);
  const float e = __fadd_rn(__fsub_rn(F, __fsub_rn(s, bb)), __fsub_rn(t, bb));
  Fc = __fadd_rn(Fc, e);
  F = s;
}

// (h, l) += x in float-float: TwoSum of h and x, then a fast renormalisation
__device__ __forceinline__ void ff_add(float &h, float &l, float x) {
  const float s = h + x;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (x - bb);
  const float t = l + e;
  const float hn = s + t;
  l = t - (hn - s);
  h = hn;
}

// coefficients of the single-precision update, read once per item into registers
struct CoefF {
  double dtVG;
  float dtK, dtcGn, Tmax, th;
};

__device__ __forceinline__ CoefF load_coef(const StepCoef *__restrict__ cf) {
  CoefF c;
  c.dtVG = cf->dtVG;
  c.dtK = cf->dtK_f;
  c.dtcGn = cf->dtcGn_f;
  c.Tmax = cf->Tmax_f;
  c.th = cf->th_ref;
  return c;
}

// where the results of one system go
struct OutPtrs {
  float *hout, *lo;
  double *A;
  const float *srcw, *pulse_f;
  int32_t *err;
  const uint8_t *fix;   // border mask (null: none)
  float2 *res;          // border reservoirs: float pairs in delta units
};

// state update of one atom (single-precision path); Ai is the atom's exchanged
// energy before this substep, F + Fc its compensated pair sum (the pair terms,
// exact negatives of each other, summed with TwoSum); returns the new hi.
// Every increment reaches the float-pair state exactly to first order: dt K F
// and the coupling term as two-float products (the rounded product, then its
// exact error), so the state's sum over atoms changes by the coupling and the
// source only, to the state's 48 bits (the rounding of each atom's own sum and
// product would otherwise add a bias to the energy of about 1e-10 per 40
// substeps on a hot system).
// BORDER: a border atom (fixed, the mask value its caller loaded with the other
// per-atom inputs) keeps its value, its change goes to o.res
template <bool LASER, bool BORDER>
__device__ __forceinline__ float update_atom(int64_t s, float di, float li, float ui, double Ai, float F, float Fc,
                                             const CoefF &cf, const OutPtrs &o, int k, bool fixed = false) {
  const float p0 = __fmul_rn(cf.dtK, F);
  float er = fmaf(cf.dtK, F, -p0);      // p0 + er == dtK * F exactly
  er = fmaf(cf.dtK, Fc, er);
  const bool chi = (ui == ui);
  float d = 0.0f, q0 = 0.0f;
  if (chi) {
    d = fmaf(cf.Tmax, di, ui);           // T_i - T_l,i
    q0 = __fmul_rn(-cf.dtcGn, d);
    er += fmaf(-cf.dtcGn, d, -q0);       // q0 + its error == -dtcGn * d exactly
  }
  float h = di, l = li;
  ff_add(h, l, p0);
  if (chi) ff_add(h, l, q0);
  ff_add(h, l, er);
  float p = 0.0f, e = 0.0f;
  if (LASER) {
    const float c = o.pulse_f[k], w = o.srcw[s];
    p = __fmul_rn(c, w);                 // not fused into the sums below
    e = fmaf(c, w, -p);                  // p + e == c * w exactly
    ff_add(h, l, p);
    ff_add(h, l, e);
  }
  if (BORDER && fixed) {
    // border atom: its value stays; the change it would have made, the increments
    // just added to the float pair, goes to its float-pair reservoir (single-
    // precision arithmetic only, as exact as the state)
    float2 r = o.res[s];
    ff_add(r.x, r.y, p0);
    if (chi) ff_add(r.x, r.y, q0);
    ff_add(r.x, r.y, er);
    if (LASER) {
      ff_add(r.x, r.y, p);
      ff_add(r.x, r.y, e);
    }
    o.res[s] = r;
    h = di;
    l = li;
  }
  o.hout[s] = h;
  o.lo[s] = l;
  if (chi) o.A[s] = fma(cf.dtVG, f2d(d), Ai);
  const float th = cf.th + h;
  if (!(th >= 0.0f && th <= 1.0f)) atomicOr(o.err, ERR_RANGE);
  return h;
}

// LOCAL form, state update of one atom (single-precision paths): (h, l) is the
// float pair of w = u - u_ref, F + Fc the compensated pair sum; the new mirror
// value delta = theta - theta_ref goes to hout[s] and is returned
__device__ __forceinline__ float update_atom_local(int64_t s, float di, float h, float l, float ui, double Ai,
                                                   float F, float Fc, const StepCoef *__restrict__ cf,
                                                   float *__restrict__ hout, float *__restrict__ uhi,
                                                   float *__restrict__ lo, double *__restrict__ A,
                                                   int32_t *__restrict__ err) {
  const float th = cf->th_ref;
  const float Ku = cf->dtKu_f;
  const float p0 = __fmul_rn(Ku, F);
  ff_add(h, l, p0);
  ff_add(h, l, fmaf(Ku, F, -p0) + Ku * Fc);     // the product's error and the compensation
  const bool chi = (ui == ui);
  float dT = 0.0f;
  if (chi) {
    dT = fmaf(cf->Tmax_f, di, ui);               // T_i - T_l,i
    const float g = -cf->dtgu_f;
    const float q0 = __fmul_rn(g, dT);
    ff_add(h, l, q0);
    ff_add(h, l, fmaf(g, dT, -q0));
  }
  uhi[s] = h;
  lo[s] = l;
  if (chi) A[s] = fma(cf->dtVGu, f2d(dT), Ai);
  float dn;
  if (cf->thc_f > 0.0f && h > cf->wc_f) {
    dn = fmaf(h - cf->wc_f, cf->inv_thc_f, cf->thc_f - th);
  } else {
    const float q = fmaf(2.0f, h, cf->thsq_f);
    dn = (2.0f * h) / (sqrtf(q) + th);
  }
  hout[s] = dn;
  const float tn = th + dn;
  if (!(tn >= 0.0f && tn <= 1.0f)) atomicOr(err, ERR_RANGE);
  return dn;
}

// Tile descriptor of the row tile around row R of one system.  Neighbour row r
// is placed at tile offset off[r]: after the previous row rounded up to 4
// words, congruent to its first global index modulo 4, so that each row moves
// as one 16-byte aligned bulk copy of its aligned superset.  The system's
// arguments are copied next to it, so every warp reads them from shared memory.
struct TileDesc {
  int32_t start[kRowNbr], len[kRowNbr], off[kRowNbr];
  int32_t self_base, row_s, row_len, tier, row;
  int32_t staged;   // words the tile occupies
  int32_t pad[2];
  RepArgs ra;
  StepCoef cf;      // the system's step coefficients (a copy, read from shared memory)
};

// computed by one warp: lane r < 9 handles neighbour row r
// rr_in: row ranges to read instead of the system's own (null: the system's)
__device__ __forceinline__ void make_desc(const RepArgs *__restrict__ reps, int2 item, int parity, TileDesc *d,
                                          const float *rr_in = nullptr) {
  const int lane = threadIdx.x & 31;
  // copy the system's arguments (whole 8-byte words) into the descriptor
  static_assert(sizeof(RepArgs) % 8 == 0, "RepArgs must be a whole number of 8-byte words");
  const uint64_t *src = reinterpret_cast<const uint64_t *>(reps + item.x);
  uint64_t *dst = reinterpret_cast<uint64_t *>(&d->ra);
  for (int w = lane; w < (int)(sizeof(RepArgs) / 8); w += 32) dst[w] = __ldg(src + w);
  __syncwarp();
  static_assert(sizeof(StepCoef) % 8 == 0, "StepCoef must be a whole number of 8-byte words");
  {
    const uint64_t *cs = reinterpret_cast<const uint64_t *>(d->ra.cf);
    uint64_t *cd = reinterpret_cast<uint64_t *>(&d->cf);
    for (int w = lane; w < (int)(sizeof(StepCoef) / 8); w += 32) cd[w] = __ldg(cs + w);
  }
  const int R = item.y;
  const int32_t ncx = d->ra.ncx;
  const int32_t *row_nbr = d->ra.row_nbr;
  const int32_t *start = d->ra.start;
  const float *rr = rr_in ? rr_in : d->ra.rrange[parity];
  const int32_t nrows = d->ra.nrows;
  int32_t R2 = -1, a = 0, len = 0;
  float mn = 3.0e38f, mx = -3.0e38f;
  if (lane < kRowNbr) {
    R2 = __ldg(row_nbr + (int64_t)R * kRowNbr + lane);
    if (R2 >= 0) {
      a = __ldg(start + (int64_t)R2 * ncx);
      len = __ldg(start + (int64_t)R2 * ncx + ncx) - a;
      mn = rr[R2];
      mx = rr[nrows + R2];
    }
  }
  // placement, sequential over the 9 rows (same rule as the neighbour build)
  int32_t off = 0, end = 0;
  for (int r = 0; r < kRowNbr; ++r) {
    const int32_t ar = __shfl_sync(0xffffffffu, a, r);
    const int32_t lr = __shfl_sync(0xffffffffu, len, r);
    const int32_t o = ((end + 3) & ~3) + (ar & 3);
    if (lane == r) off = o;
    end = o + lr;
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const unsigned selfm = __ballot_sync(0xffffffffu, R2 == R);
  const int sl = __ffs(selfm) - 1;
  if (lane < kRowNbr) {
    d->start[lane] = a;
    d->len[lane] = len;
    d->off[lane] = off;
  }
  if (lane == sl) {
    d->self_base = off;
    d->row_s = a;
    d->row_len = len;
    d->row = R;
    d->staged = (end + 3) & ~3;
    const float spread = mx - mn;
    d->tier = spread < 1.2e-4f ? 3 : (spread < 0.02f ? 2 : (spread < 0.12f ? 1 : 0));
  }
  __syncwarp();
}

// ---- mbarrier and bulk-copy primitives (CTA scope) ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
// arrive once and add `bytes` to the transaction count of the current phase
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the completion of the phase with the given parity; gives up (false)
// after a bounded number of polls, each of which may suspend the thread briefly
constexpr uint32_t kMaxPolls = 1u << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
  for (uint32_t i = 0; i < kMaxPolls; ++i)
    if (mbar_test(b, parity)) return true;
  return false;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
// that completes `bytes` transactions on barrier `bar`
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Failure-detection probe: the bounded wait of the tile kernels on an mbarrier
// phase that completes (count 1, one arrival) or never completes (count 2, one
// arrival: a flag nothing sets).  After `polls` unsuccessful polls the block
// records ERR_TIMEOUT in *flag and returns; no asynchronous copy is involved.
__global__ void wait_probe_kernel(uint32_t polls, int complete, int32_t *__restrict__ flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, complete ? 1u : 2u);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive(&bar);
  bool ok = false;
  for (uint32_t i = 0; i < polls && !ok; ++i) ok = mbar_test(&bar, 0);
  if (!ok) atomicOr(flag, ERR_TIMEOUT);
}

// per-atom inputs of a Chebyshev stage
struct StageIn {
  float zm1, zm2, y0, F0;
};

// LOCAL: the LOCAL C_e / kappa_e form (wh: the high word of the atom's energy
// state, li its low word): the series order TIER is the one of the whole
// substep (a per-tile order could differ between the two tiles a pair spans, and
// the pair terms must be exact negatives), kappa_ij weights, TwoSum sums; the
// largest |Delta| seen is raised in *mdp
template <int TIER, bool LASER, int PP, bool STAGE, bool BORDER, bool LOCAL = false>
__device__ __forceinline__ float row_atom(const RepArgs &ra, const StepCoef *cf, const StageArgs &sa, int parity,
                                          int k, const float *tile, uint32_t tlen, int32_t s, float di,
                                          const uint32_t *pv, float ui, float li, double Ai, const StageIn &si,
                                          bool fixed, float wh = 0.0f, float *mdp = nullptr) {
  const float th = cf->th_ref;
  const float ai = th + di;
  const float m2ai = -2.0f * ai;
  if (LOCAL) {
    const bool km = cf->kmode != 0;
    float F = 0.0f, Fc = 0.0f;
#pragma unroll
    for (int m = 0; m < PP; ++m)
      if (PP != 16 || m < ra.P) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const float dj = tile[checked_index(half ? (pv[m] >> 16) : (pv[m] & 0xffffu), tlen, ra.err)];
          const float fij = pair_acc<TIER>(0.0f, di, dj, th, ai, m2ai);
          const float kij = km ? 0.5f * (ai + (th + dj)) : 1.0f;
          two_sum_acc(F, Fc, __fmul_rn(kij, fij));
          *mdp = fmaxf(*mdp, fabsf(dj - di));
        }
      }
    return update_atom_local(s, di, wh, li, ui, Ai, F, Fc, cf, ra.dmir[parity ^ 1], ra.uhi, ra.lo, ra.A, ra.err);
  }
  float F = 0.0f, Fc = 0.0f;
  if (STAGE) {
#pragma unroll
    for (int m = 0; m < PP; ++m)
      if (PP != 16 || m < ra.P) {
        F = pair_acc<TIER>(F, di, tile[checked_index(pv[m] & 0xffffu, tlen, ra.err)], th, ai, m2ai);
        F = pair_acc<TIER>(F, di, tile[checked_index(pv[m] >> 16, tlen, ra.err)], th, ai, m2ai);
      }
  } else {
    // the pair terms (exact negatives of their partners' terms), compensated sum
#pragma unroll
    for (int m = 0; m < PP; ++m)
      if (PP != 16 || m < ra.P) {
        two_sum_acc(F, Fc, pair_flux<TIER>(di, tile[checked_index(pv[m] & 0xffffu, tlen, ra.err)], th, ai, m2ai));
        two_sum_acc(F, Fc, pair_flux<TIER>(di, tile[checked_index(pv[m] >> 16, tlen, ra.err)], th, ai, m2ai));
      }
  }
  if (STAGE) {
    // Chebyshev stage on the window's change: z_j = z_{j-1} + nu (z_{j-2} - z_{j-1})
    // - kap z_{j-1} + mut tau K F(Y_{j-1}) + gam tau K F(Y_0), Y_j = Y_0 + z_j
    const float inc = fmaf(sa.gt, si.F0, fmaf(-sa.kap, si.zm1, sa.mt * F));
    const float z = si.zm1 + fmaf(sa.nu, si.zm2 - si.zm1, inc);
    const float h = si.y0 + z;
    float hw = h;
    if (sa.T1) {   // the last stage: the window's end in FP64 and its coupling
      const double t0 = sa.T0[s];
      const float ui = ra.uTl[s];
      float dT = 0.0f;
      if (ui == ui) dT = sa.fin * ((d2f_rn(t0) - sa.Tref_f) + ui);   // fin (T0 - T_l), T_l = Tref - ui
      const double dTd = f2d(dT);
      sa.T1[s] = fma(sa.Tmax, f2d(z), t0) - dTd;
      sa.dTc[s] = dTd;
      if (dT != 0.0f) hw = fmaf(-dT, sa.invTmax_f, h);
    }
    if (sa.zout) {   // null: a flux pass, whose stage values are not kept
      sa.zout[s] = z;
      sa.yout[s] = hw;
    }
    if (sa.Fout) sa.Fout[s] = F;
    return h;
  }
  const OutPtrs o = {ra.dmir[parity ^ 1], ra.lo, ra.A, ra.srcw, ra.pulse_f, ra.err, ra.fix,
                     reinterpret_cast<float2 *>(ra.res)};
  return update_atom<LASER, BORDER>(s, di, li, ui, Ai, F, Fc, load_coef(cf), o, k, fixed);
}

constexpr int kTileBufs = 2;   // tiles in flight per CTA
constexpr int kDescAhead = 2;  // descriptors are prepared this many items ahead of their copies
constexpr int kDescRing = kTileBufs + kDescAhead + 1;

template <int NT>
struct TilePipe {
  uint64_t full[kTileBufs];    // tile b holds its item (one arrival + the copied bytes)
  uint64_t empty[kTileBufs];   // every compute warp is done with tile b
  TileDesc desc[kDescRing];    // item it uses slot it % kDescRing
  float wmin[kTileBufs][NT / 32], wmax[kTileBufs][NT / 32];
};

// producer side, after the compute warps released tile b of item it: the row's
// value range for the tier choice of the next substep
template <int NT>
__device__ __forceinline__ void close_item(TilePipe<NT> &sp, int it, int parity, float *rr_out = nullptr) {
  const int b = it % kTileBufs;
  if ((threadIdx.x & 31) == 0) {
    float a = sp.wmin[b][0], c = sp.wmax[b][0];
    for (int w = 1; w < NT / 32; ++w) {
      a = fminf(a, sp.wmin[b][w]);
      c = fmaxf(c, sp.wmax[b][w]);
    }
    const TileDesc &D = sp.desc[it % kDescRing];
    float *rr = rr_out ? rr_out : D.ra.rrange[parity ^ 1];
    rr[D.row] = a;
    rr[D.ra.nrows + D.row] = c;
  }
  __syncwarp();
}

// Persistent row-tile kernel over a work list of (system, row) items; CTA c
// takes items c, c + gridDim.x, ...  Warp-specialised pipeline on two tile
// buffers: the last warp writes each item's descriptor (two items ahead, so its
// chain of dependent loads is off the critical path) and fetches the item's 9
// rows with bulk copies as soon as a buffer frees (one lane, completion counted
// on full[b]); the compute warps
// wait on full[b], sweep the row's atoms and arrive on empty[b], which the
// producer waits for before reusing the buffer.  No CTA-wide barrier inside the
// loop, so fast warps run ahead by up to one item.  Every wait is bounded: on
// a timeout the warp records ERR_TIMEOUT and stops, and the producer waits
// (bounded) for its copies in flight before leaving.
// PP = 9: exactly nine index words per atom (18-neighbour FCC shells) in every
// system; PP = 16: any count up to 32 neighbours, ra.P words.
// STAGE: one stage of the Chebyshev window propagator instead of a substep
// (pair flux of the tile values sa.yin, stage update into sa.yout, optionally
// the flux itself into sa.Fout); rows and tiers as for substeps.
// NT: threads that own atoms (256, or 128 for short rows); one producer warp more.
template <bool LASER, int PP, bool STAGE, int NT, bool BORDER = false, bool LOCAL = false>
__global__ void __launch_bounds__(NT + 32, NT == 256 ? kTileMinBlocks : 2 * kTileMinBlocks)
    substep_tile_kernel(const RepArgs *__restrict__ reps, const int2 *__restrict__ work, int32_t nwork, int32_t tb,
                        int parity, int k, StageArgs sa) {
  extern __shared__ __align__(128) float tiles[];   // kTileBufs x tb words
  __shared__ TilePipe<NT> sp;
  if ((int)blockIdx.x >= nwork) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int aw = NT / 32;   // warps 0..aw-1 compute; warp aw produces
  const int n_it = (nwork - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  if (threadIdx.x == 0) {
    for (int b = 0; b < kTileBufs; ++b) {
      mbar_init(&sp.full[b], 1);
      mbar_init(&sp.empty[b], aw);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  if (warp == aw) {
    int32_t *err = nullptr;
    int issued = 0;
    bool ok = true;
    const float *rr_in = STAGE ? sa.rr[parity] : nullptr;
    float *rr_out = STAGE ? sa.rr[parity ^ 1] : nullptr;
    make_desc(reps, work[blockIdx.x], parity, &sp.desc[0], rr_in);
    int made = 1;
    for (int it = 0; it < n_it && ok; ++it) {
      const int b = it % kTileBufs;
      const uint32_t use = (uint32_t)(it / kTileBufs);
      if (use > 0) {
        ok = mbar_wait(&sp.empty[b], (use - 1) & 1);
        if (!ok) break;
        close_item(sp, it - kTileBufs, parity, rr_out);
      }
      TileDesc *d = &sp.desc[it % kDescRing];
      err = d->ra.err;
      if (lane == 0) {
        const float *hin = STAGE ? sa.yin : d->ra.dmir[parity];
        float *dst = tiles + (int64_t)b * tb;
        // an empty row has nothing to update (and its tile is not covered by
        // the build's largest-tile figure): copy nothing.  A row whose tile
        // exceeds the buffer cannot occur after a build; if it did, it is
        // skipped and reported.
        if (d->row_len > 0 && d->staged > tb) {
          atomicOr(d->ra.err, ERR_NBR_OVERFLOW);
          d->row_len = 0;
        }
        const bool copy = d->row_len > 0;
        uint32_t bytes = 0;
        for (int r = 0; r < kRowNbr && copy; ++r) {
          const int32_t a = d->start[r], len = d->len[r];
          if (len > 0) bytes += (uint32_t)(((a + len + 3) & ~3) - (a & ~3)) * 4u;
        }
        mbar_arrive_expect(&sp.full[b], bytes);
        for (int r = 0; r < kRowNbr && copy; ++r) {
          const int32_t a = d->start[r], len = d->len[r];
          if (len <= 0) continue;
          const int32_t a0 = a & ~3, a1 = (a + len + 3) & ~3;
          bulk_copy(dst + (d->off[r] - (a & 3)), hin + a0, (uint32_t)(a1 - a0) * 4u, &sp.full[b]);
        }
      }
      __syncwarp();
      issued = it + 1;
      // descriptors ahead: one after the first item's copies, then up to kDescAhead
      const int want = (it == 0) ? 2 : it + 1 + kDescAhead;
      for (; made < want && made < n_it; ++made)
        make_desc(reps, work[blockIdx.x + (int64_t)made * gridDim.x], parity, &sp.desc[made % kDescRing],
                  rr_in);
    }
    // release the last items: their row ranges
    for (int it = (issued > kTileBufs ? issued - kTileBufs : 0); it < issued && ok; ++it) {
      ok = mbar_wait(&sp.empty[it % kTileBufs], (uint32_t)(it / kTileBufs) & 1);
      if (ok) close_item(sp, it, parity, rr_out);
    }
    if (!ok) {
      if (lane == 0 && err) atomicOr(err, ERR_TIMEOUT);
      // no copy may still be landing when the CTA leaves
      for (int it = (issued > kTileBufs ? issued - kTileBufs : 0); it < issued; ++it)
        mbar_wait(&sp.full[it % kTileBufs], (uint32_t)(it / kTileBufs) & 1);
    }
    return;
  }
  // compute warps
  // LOCAL form: one series order for the substep, from the previous substep's
  // largest |Delta| (margin 1.25; the first substep of a call: the full series)
  int ltier = 0;
  float lmd = 0.0f;
  if (LOCAL) {
    uint32_t *ring = reps[0].ldmax;
    const float prev = 1.25f * __uint_as_float(ring[k % 3]);
    ltier = prev < 1.2e-4f ? 3 : (prev < 0.02f ? 2 : (prev < 0.12f ? 1 : 0));
    if (blockIdx.x == 0 && threadIdx.x == 0) ring[(k + 2) % 3] = 0u;
  }
  // The atoms of a row go to the compute warps in rounds of NT; the warps that
  // take a row's last, partial round rotate from row to row (rot: the first of
  // them), so that no warp carries every row's extra round and holds the others,
  // which run at most one item ahead, back.
  int rot = 0;
  for (int it = 0; it < n_it; ++it) {
    const int b = it % kTileBufs;
    if (!mbar_wait(&sp.full[b], (uint32_t)(it / kTileBufs) & 1)) {
      if (lane == 0) atomicOr(reps[0].err, ERR_TIMEOUT);
      return;
    }
    const TileDesc &D = sp.desc[it % kDescRing];
    const int row_len = D.row_len, row_s = D.row_s, sb = D.self_base;
    const int tier = D.tier;
    const float *tile = tiles + (int64_t)b * tb;
    const int64_t ps = D.ra.ps;
    const uint32_t *pidx = D.ra.pidx;
    float vmin = 3.0e38f, vmax = -3.0e38f;
    const int vw = (warp + aw - rot) % aw;   // this warp's place in the row's rounds
    for (int q = vw * 32 + lane; q < row_len; q += NT) {
      const int32_t s = row_s + q;
      uint32_t pv[PP];
#pragma unroll
      for (int m = 0; m < PP; ++m)
        if (PP != 16 || m < D.ra.P) pv[m] = __ldg(pidx + (m * ps + s));
      const float di = tile[sb + q];
      float ui = 0.0f, li = 0.0f, wh = 0.0f;
      double Ai = 0.0;
      bool fixed = false;
      StageIn si = {0.0f, 0.0f, 0.0f, 0.0f};
      if (STAGE) {
        si.y0 = sa.y0[s];
        if (sa.zin) si.zm1 = sa.zin[s];
        if (sa.zprev) si.zm2 = sa.zprev[s];
        if (sa.F0) si.F0 = sa.F0[s];
      } else {
        ui = D.ra.uTl[s];
        li = D.ra.lo[s];
        Ai = D.ra.A[s];
        if (BORDER) fixed = D.ra.fix[s] != 0;
        if (LOCAL) wh = D.ra.uhi[s];
      }
      float h;
      if (LOCAL) {
        const uint32_t tl = (uint32_t)D.staged;
        if (ltier == 3) h = row_atom<3, false, PP, false, false, true>(D.ra, &D.cf, sa, parity, k, tile, tl, s, di, pv, ui, li, Ai, si, false, wh, &lmd);
        else if (ltier == 2) h = row_atom<2, false, PP, false, false, true>(D.ra, &D.cf, sa, parity, k, tile, tl, s, di, pv, ui, li, Ai, si, false, wh, &lmd);
        else if (ltier == 1) h = row_atom<1, false, PP, false, false, true>(D.ra, &D.cf, sa, parity, k, tile, tl, s, di, pv, ui, li, Ai, si, false, wh, &lmd);
        else h = row_atom<0, false, PP, false, false, true>(D.ra, &D.cf, sa, parity, k, tile, tl, s, di, pv, ui, li, Ai, si, false, wh, &lmd);
      }
      else if (tier == 3) h = row_atom<3, LASER, PP, STAGE, BORDER>(D.ra, &D.cf, sa, parity, k, tile, (uint32_t)D.staged, s, di, pv, ui, li, Ai,
                                                              si, fixed);
      else if (tier == 2) h = row_atom<2, LASER, PP, STAGE, BORDER>(D.ra, &D.cf, sa, parity, k, tile, (uint32_t)D.staged, s, di, pv, ui, li, Ai,
                                                                   si, fixed);
      else if (tier == 1) h = row_atom<1, LASER, PP, STAGE, BORDER>(D.ra, &D.cf, sa, parity, k, tile, (uint32_t)D.staged, s, di, pv, ui, li, Ai,
                                                                   si, fixed);
      else h = row_atom<0, LASER, PP, STAGE, BORDER>(D.ra, &D.cf, sa, parity, k, tile, (uint32_t)D.staged, s, di, pv, ui, li, Ai,
                                                    si, fixed);
      vmin = fminf(vmin, h);
      vmax = fmaxf(vmax, h);
    }
    for (int o = 16; o > 0; o >>= 1) {
      vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
      vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if (lane == 0) {
      sp.wmin[b][warp] = vmin;
      sp.wmax[b][warp] = vmax;
      mbar_arrive(&sp.empty[b]);
    }
    __syncwarp();
    rot = (rot + ((row_len % NT) + 31) / 32) % aw;
  }
  if (LOCAL) {
    for (int o = 16; o > 0; o >>= 1) lmd = fmaxf(lmd, __shfl_xor_sync(0xffffffffu, lmd, o));
    if (lane == 0) {
      uint32_t *nx = reps[0].ldmax + (k + 1) % 3;
      const uint32_t mb = __float_as_uint(lmd);
      if (mb > *((volatile uint32_t *)nx)) atomicMax(nx, mb);
    }
  }
}

// general single-precision path: one thread per atom, int32 neighbour table,
// neighbour values gathered from global memory (any row length)
template <bool LASER>
// wgt (if not null): pair weights w_ij [slot][atom] multiplying each pair term
__global__ void __launch_bounds__(256) substep_f32_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt,
    const float *__restrict__ hin, float *__restrict__ hout, float *__restrict__ lo, double *__restrict__ A,
    const float *__restrict__ uTl, const float *__restrict__ srcw, const float *__restrict__ pulse_f, int k,
    const StepCoef *__restrict__ cf, int32_t *__restrict__ err, const float *__restrict__ wgt,
    const uint8_t *__restrict__ fix, double *__restrict__ res) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float th = cf->th_ref;
  const int c = cnt[s];
  const float di = hin[s];
  const bool fixed = fix && fix[s];
  const float ai = th + di, m2ai = -2.0f * ai;
  // pair terms (exact negatives of their partners' terms, the weights symmetric)
  // summed with TwoSum
  float F = 0.0f, Fc = 0.0f;
  const int32_t *np = nbr + s;
  int j = 0;
  if (wgt) {
    // six pairs at a time: their index, weight and value loads are in flight together
    const float *wp = wgt + s;
    for (; j + 6 <= c; j += 6) {
      int32_t t[6];
      float dj[6], wj[6];
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        t[u] = checked_index(__ldg(np + (int64_t)(j + u) * n), n, err);
        wj[u] = __ldg(wp + (int64_t)(j + u) * n);
      }
#pragma unroll
      for (int u = 0; u < 6; ++u) dj[u] = __ldg(hin + t[u]);
#pragma unroll
      for (int u = 0; u < 6; ++u) two_sum_acc(F, Fc, __fmul_rn(wj[u], pair_term(di, dj[u], th, ai, m2ai)));
    }
    for (; j < c; ++j)
      two_sum_acc(F, Fc, __fmul_rn(__ldg(wp + (int64_t)j * n),
                                   pair_term(di, __ldg(hin + checked_index(__ldg(np + (int64_t)j * n), n, err)),
                                             th, ai, m2ai)));
  }
  for (; j + 6 <= c; j += 6) {
    int32_t t[6];
    float dj[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) t[u] = checked_index(__ldg(np + (int64_t)(j + u) * n), n, err);
#pragma unroll
    for (int u = 0; u < 6; ++u) dj[u] = __ldg(hin + t[u]);
#pragma unroll
    for (int u = 0; u < 6; ++u) two_sum_acc(F, Fc, pair_term(di, dj[u], th, ai, m2ai));
  }
  for (; j < c; ++j)
    two_sum_acc(F, Fc, pair_term(di, __ldg(hin + checked_index(__ldg(np + (int64_t)j * n), n, err)), th, ai, m2ai));
  const OutPtrs o = {hout, lo, A, srcw, pulse_f, err, fix, reinterpret_cast<float2 *>(res)};
  update_atom<LASER, true>(s, di, lo[s], uTl[s], A[s], F, Fc, load_coef(cf), o, k, fixed);
}

// Pair sum of the LOCAL form for one atom with the series order TIER (one order
// for every atom of the substep, so the two terms of a pair stay exact negatives);
// also the largest |Delta| seen
template <int TIER>
__device__ __forceinline__ void local_pair_sum(int32_t n, int32_t s, int c, const int32_t *__restrict__ nbr,
                                               const float *__restrict__ hin, const float *__restrict__ wgt,
                                               float di, float th, float ai, float m2ai, bool km,
                                               int32_t *__restrict__ err, float &F, float &Fc, float &md) {
  const int32_t *np = nbr + s;
  const float *wp = wgt ? wgt + s : nullptr;
  int j = 0;
  for (; j + 6 <= c; j += 6) {
    int32_t t[6];
    float dj[6], wj[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      t[u] = checked_index(__ldg(np + (int64_t)(j + u) * n), n, err);
      wj[u] = wp ? __ldg(wp + (int64_t)(j + u) * n) : 1.0f;
    }
#pragma unroll
    for (int u = 0; u < 6; ++u) dj[u] = __ldg(hin + t[u]);
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const float fij = pair_acc<TIER>(0.0f, di, dj[u], th, ai, m2ai);
      const float kij = km ? 0.5f * (ai + (th + dj[u])) : 1.0f;
      two_sum_acc(F, Fc, __fmul_rn(__fmul_rn(kij, wj[u]), fij));
      md = fmaxf(md, fabsf(dj[u] - di));
    }
  }
  for (; j < c; ++j) {
    const float dj = __ldg(hin + checked_index(__ldg(np + (int64_t)j * n), n, err));
    const float wj = wp ? __ldg(wp + (int64_t)j * n) : 1.0f;
    const float fij = pair_acc<TIER>(0.0f, di, dj, th, ai, m2ai);
    const float kij = km ? 0.5f * (ai + (th + dj)) : 1.0f;
    two_sum_acc(F, Fc, __fmul_rn(__fmul_rn(kij, wj), fij));
    md = fmaxf(md, fabsf(dj - di));
  }
}

// LOCAL per-atom C_e / kappa_e form, single precision (one thread per atom).
// Series order: one for all atoms of a substep (the two terms of every pair stay
// exact negatives), chosen from the largest |Delta| of the previous substep of
// the call, with a margin of 1.25, against the row tiles' thresholds (truncation
// below 3e-8 of B); the first substep of a call takes the full series.
// dmax[3]: the largest |Delta| as float bits, in a ring: substep k reads
// dmax[k % 3], raises dmax[(k + 1) % 3] and clears dmax[(k + 2) % 3], which no
// other substep touches meanwhile.  Choosing the order per pair instead
// (pair_term) measured slower here (133 against 128 us per substep on the 4M
// track): the branches cost more than the series they save.
// The state is each atom's electron energy density in units of gamma Tmax^2,
// held as the float pair (uhi, lo) of w = u - u_ref; hin / hout hold the mirror
// delta = theta - theta_ref the neighbours read, rebuilt from w after the update:
//   below the cap  theta = sqrt(theta_ref^2 + 2 w), delta = 2 w / (theta + theta_ref)
//   above it       theta = theta_c + (w - w_c) / theta_c
// Pair term kappa_ij f_ij with kappa_ij / kappa_scale = (theta_i + theta_j) / 2
// (kappa_mode 1) or 1: the mean is formed from fl(theta_i + theta_j), which both
// atoms compute alike, and multiplies the already rounded fl(Delta B), so the
// two atoms' terms t_ij are exact negatives.  They are summed with TwoSum (the
// sum and its rounding errors), and dt Ku times that sum enters the float-pair
// state as an exact two-float product, as does the coupling: sum_i w_i changes
// only by the second-order rounding of the compensation (single-precision
// rounding of the accumulation and of the product would leave a bias of
// about 1e-11 of the energy per substep on a hot track core).
//   w_i += dt Ku sum_j kappa_ij f_ij w_ij - chi_i dt G/(gamma Tmax^2) (T_i - T_l,i) + source
template <bool LASER>
__global__ void __launch_bounds__(256) substep_local_f32_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt,
    const float *__restrict__ hin, float *__restrict__ hout, float *__restrict__ uhi, float *__restrict__ lo,
    double *__restrict__ A, const float *__restrict__ uTl, const float *__restrict__ srcw,
    const float *__restrict__ pulse_f, int k, const StepCoef *__restrict__ cf, int32_t *__restrict__ err,
    const float *__restrict__ wgt, uint32_t *__restrict__ dmax) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) dmax[(k + 2) % 3] = 0u;
  if (s >= n) return;
  const float th = cf->th_ref;
  const bool km = cf->kmode != 0;
  const int c = cnt[s];
  const float di = hin[s];
  const float ai = th + di, m2ai = -2.0f * ai;
  float F = 0.0f, Fc = 0.0f, md = 0.0f;
  const float prev = 1.25f * __uint_as_float(dmax[k % 3]);   // the same value in every thread
  if (prev < 1.2e-4f) local_pair_sum<3>(n, s, c, nbr, hin, wgt, di, th, ai, m2ai, km, err, F, Fc, md);
  else if (prev < 0.02f) local_pair_sum<2>(n, s, c, nbr, hin, wgt, di, th, ai, m2ai, km, err, F, Fc, md);
  else if (prev < 0.12f) local_pair_sum<1>(n, s, c, nbr, hin, wgt, di, th, ai, m2ai, km, err, F, Fc, md);
  else local_pair_sum<0>(n, s, c, nbr, hin, wgt, di, th, ai, m2ai, km, err, F, Fc, md);
  {
    // raise the next substep's bound (a read first: most atoms need no atomic)
    uint32_t *nx = dmax + (k + 1) % 3;
    const uint32_t mb = __float_as_uint(md);
    if (mb > *((volatile uint32_t *)nx)) atomicMax(nx, mb);
  }
  const float Ku = cf->dtKu_f;
  const float p0 = __fmul_rn(Ku, F);
  const float e0 = fmaf(Ku, F, -p0) + Ku * Fc;   // the product's error and the compensation
  const float ui = uTl[s];
  const bool chi = (ui == ui);
  float dT = 0.0f;
  float h = uhi[s], l = lo[s];
  ff_add(h, l, p0);
  ff_add(h, l, e0);
  if (chi) {
    dT = fmaf(cf->Tmax_f, di, ui);        // T_i - T_l,i
    const float g = -cf->dtgu_f;
    const float q0 = __fmul_rn(g, dT);
    ff_add(h, l, q0);
    ff_add(h, l, fmaf(g, dT, -q0));       // exactly dt G (T_i - T_l,i) / (gamma Tmax^2) in two parts
  }
  if (LASER) {
    const float cc = pulse_f[k], w = srcw[s];
    const float p = __fmul_rn(cc, w);
    ff_add(h, l, p);
    ff_add(h, l, fmaf(cc, w, -p));        // the exact product, in two parts
  }
  uhi[s] = h;
  lo[s] = l;
  // the lattice gets what the electrons lost: the same single-precision coefficient
  if (chi) A[s] = fma(cf->dtVGu, f2d(dT), A[s]);
  float dn;
  if (cf->thc_f > 0.0f && h > cf->wc_f) {
    dn = fmaf(h - cf->wc_f, cf->inv_thc_f, cf->thc_f - th);
  } else {
    const float q = fmaf(2.0f, h, cf->thsq_f);
    dn = (2.0f * h) / (sqrtf(q) + th);    // NaN if the energy went negative
  }
  hout[s] = dn;
  const float tn = th + dn;
  if (!(tn >= 0.0f && tn <= 1.0f)) atomicOr(err, ERR_RANGE);
}

// LOCAL form, double precision: u(theta_i) + du -> theta by the closed-form inverse
template <bool LASER>
__global__ void __launch_bounds__(256) substep_local_f64_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt,
    const double *__restrict__ Tin, double *__restrict__ Tout, double *__restrict__ A,
    const double *__restrict__ Tl, const double *__restrict__ srcw, const double *__restrict__ pulse, int k,
    const StepCoef *__restrict__ cf, int32_t *__restrict__ err, const double *__restrict__ wgt) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double inv = cf->invTmax;
  const bool km = cf->kmode != 0;
  const int c = cnt[s];
  const double Ti = Tin[s];
  const double ti = Ti * inv;
  double F = 0.0;
  for (int j = 0; j < c; ++j) {
    const int32_t t = checked_index(__ldg(nbr + (int64_t)j * n + s), n, err);
    const double tj = __ldg(Tin + t) * inv;
    const bool lo = (ti < tj) || (ti == tj && s < t);
    const double a = lo ? ti : tj, b = lo ? tj : ti;
    const double E = exp(a - b);
    const double phi = b * (1.0 - a) * E - a * (1.0 - b) / E;
    const double kij = km ? 0.5 * (a + b) : 1.0;
    const double w = wgt ? __ldg(wgt + (int64_t)j * n + s) : 1.0;
    F += w * kij * (lo ? phi : -phi);
  }
  double du = cf->dtKu * F;
  const double tl = Tl[s];
  if (tl >= 0.0) {
    const double d = Ti - tl;
    du -= cf->dtgu * d;
    A[s] += cf->dtVG * d;
  }
  if (LASER) du += cf->dt * pulse[k] * srcw[s];
  const double th = ue_inv(ue_of(ti, cf->thc) + du, cf->thc);
  Tout[s] = th / inv;
  if (!(th >= 0.0 && th <= 1.0)) atomicOr(err, ERR_RANGE);
}

// LOCAL form: T (FP64) -> the state w = u(theta) - u_ref as a float pair and the mirror
__global__ void split_local_kernel(int64_t n, const double *__restrict__ T, double Tref, double invTmax,
                                   double thc, double u_ref, float *__restrict__ mir, float *__restrict__ uhi,
                                   float *__restrict__ lo) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double w = ue_of(T[s] * invTmax, thc) - u_ref;
  const float h = (float)w;
  uhi[s] = h;
  lo[s] = (float)(w - (double)h);
  mir[s] = (float)((T[s] - Tref) * invTmax);
}

// LOCAL form: state -> T (FP64)
__global__ void merge_local_kernel(int64_t n, const float *__restrict__ uhi, const float *__restrict__ lo,
                                   double thc, double u_ref, double Tmax, double *__restrict__ T) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  T[s] = Tmax * ue_inv(u_ref + ((double)uhi[s] + (double)lo[s]), thc);
}

// T (FP64) -> hi + lo of delta = (T - Tref) / Tmax (split_pair: the conversions on the integer pipes)
__global__ void split_kernel(int64_t n, const double *__restrict__ T, double Tref, double invTmax,
                             float *__restrict__ hi, float *__restrict__ lo) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  float h, l;
  split_pair((T[s] - Tref) * invTmax, h, l);
  hi[s] = h;
  lo[s] = l;
}

// hi + lo -> T (FP64)
__global__ void merge_kernel(int64_t n, const float *__restrict__ hi, const float *__restrict__ lo, double Tref,
                             double Tmax, double *__restrict__ T) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  T[s] = Tref + Tmax * (f2d(hi[s]) + f2d(lo[s]));   // the pair's sum is exact in FP64
}

template <bool LASER>
__global__ void __launch_bounds__(256) substep_f64_kernel(
    int32_t n, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ cnt,
    const double *__restrict__ Tin, double *__restrict__ Tout, double *__restrict__ A,
    const double *__restrict__ Tl, const double *__restrict__ srcw, const double *__restrict__ pulse,
    int k, const StepCoef *__restrict__ cf, int32_t *__restrict__ err, const double *__restrict__ wgt,
    const uint8_t *__restrict__ fix, double *__restrict__ res) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double inv = cf->invTmax;
  const int c = cnt[s];
  const double Ti = Tin[s];
  const double ti = Ti * inv;
  double F = 0.0;
  for (int j = 0; j < c; ++j) {
    const int32_t t = checked_index(__ldg(nbr + (int64_t)j * n + s), n, err);
    const double tj = __ldg(Tin + t) * inv;
    const bool lo = (ti < tj) || (ti == tj && s < t);
    const double a = lo ? ti : tj, b = lo ? tj : ti;
    const double E = exp(a - b);
    const double phi = b * (1.0 - a) * E - a * (1.0 - b) / E;
    const double w = wgt ? __ldg(wgt + (int64_t)j * n + s) : 1.0;
    F += w * (lo ? phi : -phi);
  }
  double inc = cf->dtTK * F;
  const double tl = Tl[s];
  if (tl >= 0.0) {
    const double d = Ti - tl;
    inc -= cf->dtcG * d;
    A[s] += cf->dtVG * d;
  }
  if (LASER) inc += cf->dt * pulse[k] * srcw[s];
  double To = Ti + inc;
  if (fix && fix[s]) {
    // border atom: its temperature stays, the change goes to its reservoir (kelvin)
    res[s] += To - Ti;
    To = Ti;
  }
  Tout[s] = To;
  const double th = To * inv;
  if (!(th >= 0.0 && th <= 1.0)) atomicOr(err, ERR_RANGE);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_wait_probe(uint32_t polls, int complete, int32_t *flag, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(polls, complete, flag);
  return cudaGetLastError();
}

// the row-tile kernel applies when two buffers fit in shared memory and the
// table holds at most 32 neighbours per atom
static bool tile_fits(const Ctx &c) {
  const int w = ((c.n_max + 1) / 2 == 9) ? 0 : 1;
  return c.p.flux_prec == 0 && c.p.rate_shell_n == 0 && c.W <= 32 && c.nwork > 0 &&
         c.staged_max <= c.tile_floats && c.tile_grid[w] > 0;
}

bool tile_path(const Ctx &c) { return !c.local && tile_fits(c); }

bool local_tile(const Ctx &c) { return c.local && !(c.p.laser_on && c.have_depth) && tile_fits(c); }

cudaError_t launch_split(Ctx &c, cudaStream_t st) {
  if (c.n > 0 && c.local) {
    const StepCoef &cf = *c.coef_host;
    split_local_kernel<<<nblk(c.n, 256), 256, 0, st>>>(c.n, c.T[c.tcur], c.p.Tref_K, 1.0 / c.p.Tmax_K, cf.thc,
                                                       cf.u_ref, c.dmir[c.parity], c.uhi, c.dlo);
    return cudaGetLastError();
  }
  if (c.n > 0)
    split_kernel<<<nblk(c.n, 256), 256, 0, st>>>(c.n, c.T[c.tcur], c.p.Tref_K, 1.0 / c.p.Tmax_K, c.dmir[c.parity],
                                                 c.dlo);
  return cudaGetLastError();
}

cudaError_t launch_merge(Ctx &c, int parity, cudaStream_t st) {
  if (c.n > 0 && c.local) {
    const StepCoef &cf = *c.coef_host;
    merge_local_kernel<<<nblk(c.n, 256), 256, 0, st>>>(c.n, c.uhi, c.dlo, cf.thc, cf.u_ref, c.p.Tmax_K,
                                                       c.T[c.tcur]);
    return cudaGetLastError();
  }
  if (c.n > 0)
    merge_kernel<<<nblk(c.n, 256), 256, 0, st>>>(c.n, c.dmir[parity], c.dlo, c.p.Tref_K, c.p.Tmax_K, c.T[c.tcur]);
  return cudaGetLastError();
}

// the first substep of a call takes the full series (state changed between
// calls: hand-over, stopping, a new build): the ring's first word at a large
// float (bytes 0x7f), the others cleared
static void local_tier_reset(Ctx &c, cudaStream_t st) {
  cudaMemsetAsync(c.ldmax, 0x7f, sizeof(uint32_t), st);
  cudaMemsetAsync(c.ldmax + 1, 0, 2 * sizeof(uint32_t), st);
}

// substep k of the current call; parity selects the mirror (FP32) or the T
// buffer (FP64) that holds the previous snapshot.
cudaError_t launch_substep(Ctx &c, int k, int parity, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  const int32_t n = (int32_t)c.n;
  const bool laser = c.p.laser_on && c.have_depth;
  if (c.local) {
    if (local_tile(c)) {
      if (k == 0) local_tier_reset(c, st);
      const int32_t P = (c.n_max + 1) / 2;
      const int32_t tb = c.tile_floats;
      const size_t shm = sizeof(float) * kTileBufs * (size_t)tb;
      const int32_t tg = c.tile_grid[P == 9 ? 0 : 1];
      const unsigned grid = (unsigned)(c.nwork < tg ? c.nwork : tg);
      const unsigned nt = kTileThreads + 32;
      const StageArgs none{};
      if (P == 9) substep_tile_kernel<false, 9, false, 256, false, true><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
      else substep_tile_kernel<false, 16, false, 256, false, true><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
      return cudaGetLastError();
    }
    if (c.p.flux_prec == 1) {
      const double *Tin = c.T[parity];
      double *Tout = c.T[parity ^ 1];
      if (laser)
        substep_local_f64_kernel<true><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, Tin, Tout, c.A, c.Tl_d,
                                                                     c.srcw_d, c.pulse, k, c.coef, c.err, c.wgt_d);
      else
        substep_local_f64_kernel<false><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, Tin, Tout, c.A, c.Tl_d,
                                                                      c.srcw_d, c.pulse, k, c.coef, c.err, c.wgt_d);
    } else if (laser) {
      if (k == 0) local_tier_reset(c, st);
      substep_local_f32_kernel<true><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, c.dmir[parity],
                                                                   c.dmir[parity ^ 1], c.uhi, c.dlo, c.A, c.uTl,
                                                                   c.srcw, c.pulse_f, k, c.coef, c.err, c.wgt,
                                                                   c.ldmax);
    } else {
      if (k == 0) local_tier_reset(c, st);
      substep_local_f32_kernel<false><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, c.dmir[parity],
                                                                    c.dmir[parity ^ 1], c.uhi, c.dlo, c.A, c.uTl,
                                                                    c.srcw, c.pulse_f, k, c.coef, c.err, c.wgt,
                                                                    c.ldmax);
    }
    return cudaGetLastError();
  }
  if (c.p.flux_prec == 1) {
    const double *Tin = c.T[parity];
    double *Tout = c.T[parity ^ 1];
    if (laser)
      substep_f64_kernel<true><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, Tin, Tout, c.A, c.Tl_d, c.srcw_d,
                                                             c.pulse, k, c.coef, c.err, c.wgt_d, c.has_border ? c.bmask : nullptr, c.bres);
    else
      substep_f64_kernel<false><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, Tin, Tout, c.A, c.Tl_d, c.srcw_d,
                                                              c.pulse, k, c.coef, c.err, c.wgt_d, c.has_border ? c.bmask : nullptr, c.bres);
  } else if (tile_path(c)) {
    const int32_t P = (c.n_max + 1) / 2;
    const int32_t tb = c.tile_floats;
    const size_t shm = sizeof(float) * kTileBufs * (size_t)tb;
    const bool narrow = c.tile_nt == 128 && !laser && c.tile_grid128[P == 9 ? 0 : 1] > 0;
    const int32_t tg = narrow ? c.tile_grid128[P == 9 ? 0 : 1] : c.tile_grid[P == 9 ? 0 : 1];
    const unsigned grid = (unsigned)(c.nwork < tg ? c.nwork : tg);
    const StageArgs none{};
    if (c.has_border && narrow) {
      if (P == 9) substep_tile_kernel<false, 9, false, 128, true><<<grid, 160, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
      else substep_tile_kernel<false, 16, false, 128, true><<<grid, 160, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
    } else if (c.has_border) {
      // the forms that keep border atoms
      const unsigned nt = kTileThreads + 32;
      if (P == 9) {
        if (laser) substep_tile_kernel<true, 9, false, 256, true><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
        else substep_tile_kernel<false, 9, false, 256, true><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
      } else {
        if (laser) substep_tile_kernel<true, 16, false, 256, true><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
        else substep_tile_kernel<false, 16, false, 256, true><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
      }
    } else if (narrow) {
      if (P == 9) substep_tile_kernel<false, 9, false, 128><<<grid, 160, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
      else substep_tile_kernel<false, 16, false, 128><<<grid, 160, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
    } else {
      const unsigned nt = kTileThreads + 32;
      if (P == 9) {
        if (laser) substep_tile_kernel<true, 9, false, 256><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
        else substep_tile_kernel<false, 9, false, 256><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
      } else {
        if (laser) substep_tile_kernel<true, 16, false, 256><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
        else substep_tile_kernel<false, 16, false, 256><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, k, none);
      }
    }
  } else {
    if (laser)
      substep_f32_kernel<true><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, c.dmir[parity], c.dmir[parity ^ 1],
                                                             c.dlo, c.A, c.uTl, c.srcw, c.pulse_f, k, c.coef, c.err, c.wgt, c.has_border ? c.bmask : nullptr, c.bres);
    else
      substep_f32_kernel<false><<<nblk(n, 256), 256, 0, st>>>(n, c.nbr, c.cnt, c.dmir[parity], c.dmir[parity ^ 1],
                                                              c.dlo, c.A, c.uTl, c.srcw, c.pulse_f, k, c.coef,
                                                              c.err, c.wgt, c.has_border ? c.bmask : nullptr, c.bres);
  }
  return cudaGetLastError();
}

// one stage of the Chebyshev window over the context's rows (row-tile path)
cudaError_t launch_cheb_stage(Ctx &c, const StageArgs &sa, int parity, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  const int32_t P = (c.n_max + 1) / 2;
  const int32_t tb = c.tile_floats;
  const int32_t tg = c.tile_grid[P == 9 ? 0 : 1];
  const unsigned grid = (unsigned)(c.nwork < tg ? c.nwork : tg);
  const unsigned nt = kTileThreads + 32;
  const size_t shm = sizeof(float) * kTileBufs * (size_t)tb;
  if (P == 9) substep_tile_kernel<false, 9, true, 256><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, 0, sa);
  else substep_tile_kernel<false, 16, true, 256><<<grid, nt, shm, st>>>(c.reps, c.work, c.nwork, tb, parity, 0, sa);
  return cudaGetLastError();
}

// one substep of the row-tile kernel over an explicit work list (batched
// systems), nt = 256 or 128 threads owning atoms
cudaError_t launch_tile_worklist(const RepArgs *reps, const int2 *work, int32_t nwork, int32_t tb, int grid,
                                 int pairs, int parity, int k, int nt, cudaStream_t st) {
  const unsigned g = (unsigned)(nwork < grid ? nwork : grid);
  if (g == 0) return cudaSuccess;
  const size_t shm = sizeof(float) * kTileBufs * (size_t)tb;
  const StageArgs none{};
  if (nt == 128) {
    if (pairs == 9) substep_tile_kernel<false, 9, false, 128><<<g, 160, shm, st>>>(reps, work, nwork, tb, parity, k, none);
    else substep_tile_kernel<false, 16, false, 128><<<g, 160, shm, st>>>(reps, work, nwork, tb, parity, k, none);
  } else {
    const unsigned ntt = kTileThreads + 32;
    if (pairs == 9) substep_tile_kernel<false, 9, false, 256><<<g, ntt, shm, st>>>(reps, work, nwork, tb, parity, k, none);
    else substep_tile_kernel<false, 16, false, 256><<<g, ntt, shm, st>>>(reps, work, nwork, tb, parity, k, none);
  }
  return cudaGetLastError();
}

// Tile capacity with headroom for atoms drifting between cells (tiles are
// resized only when a build outgrows them), the shared-memory opt-in of every
// instance and the resident grid of each width (grid[0]: 9 index words,
// grid[1]: 16).
bool tile_size(int32_t staged, int num_sms, int32_t *tb_out, int32_t grid[2], int32_t grid128[2]) {
  const int32_t tb = ((staged + staged / 8 + 64 + 255) / 256) * 256;
  const int64_t bytes = (int64_t)sizeof(float) * kTileBufs * tb;
  if (bytes > kTileMaxBytes) return false;
  // the shared-memory limit is an attribute of the kernel function, shared by
  // every context of the process: it only ever grows, so that a context sized
  // earlier for larger tiles keeps launching after a smaller one was sized
  static std::mutex attr_mu;
  static int64_t attr_bytes = 0;
  int64_t limit;
  {
    std::lock_guard<std::mutex> lk(attr_mu);
    attr_bytes = std::max(attr_bytes, bytes);
    limit = attr_bytes;
  }
  // [width][instance]: 256-thread instances (laser, plain, stage) and 128-thread ones (plain)
  const void *inst[2][3] = {{(const void *)substep_tile_kernel<true, 9, false, 256>,
                             (const void *)substep_tile_kernel<false, 9, false, 256>,
                             (const void *)substep_tile_kernel<false, 9, true, 256>},
                            {(const void *)substep_tile_kernel<true, 16, false, 256>,
                             (const void *)substep_tile_kernel<false, 16, false, 256>,
                             (const void *)substep_tile_kernel<false, 16, true, 256>}};
  const void *inst128[2] = {(const void *)substep_tile_kernel<false, 9, false, 128>,
                            (const void *)substep_tile_kernel<false, 16, false, 128>};
  // the border forms run on the same grid (their extra CTAs, if any, wait for a
  // free slot: no CTA waits on another)
  const void *inst_border[2][3] = {{(const void *)substep_tile_kernel<true, 9, false, 256, true>,
                                    (const void *)substep_tile_kernel<false, 9, false, 256, true>,
                                    (const void *)substep_tile_kernel<false, 9, false, 128, true>},
                                   {(const void *)substep_tile_kernel<true, 16, false, 256, true>,
                                    (const void *)substep_tile_kernel<false, 16, false, 256, true>,
                                    (const void *)substep_tile_kernel<false, 16, false, 128, true>}};
  const void *inst_local[2] = {(const void *)substep_tile_kernel<false, 9, false, 256, false, true>,
                               (const void *)substep_tile_kernel<false, 16, false, 256, false, true>};
  int32_t g[2] = {0, 0}, g128[2] = {0, 0};
  for (int w = 0; w < 2; ++w) {
    int bps = 1 << 30;
    bool ok = true;
    for (int l = 0; l < 3 && ok; ++l) {
      int b = 0;
      ok = cudaFuncSetAttribute(inst[w][l], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) == cudaSuccess &&
           cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, inst[w][l], kTileThreads + 32, (size_t)bytes) ==
               cudaSuccess &&
           b > 0;
      bps = b < bps ? b : bps;
    }
    for (int l = 0; l < 3 && ok; ++l)
      ok = cudaFuncSetAttribute(inst_border[w][l], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) ==
           cudaSuccess;
    // the LOCAL form's instances run on the same grid
    if (ok)
      ok = cudaFuncSetAttribute(inst_local[w], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) ==
           cudaSuccess;
    if (ok) g[w] = bps * num_sms;
    int b = 0;
    if (cudaFuncSetAttribute(inst128[w], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, inst128[w], 160, (size_t)bytes) == cudaSuccess && b > 0)
      g128[w] = b * num_sms;
  }
  cudaGetLastError();
  if (g[0] == 0 && g[1] == 0) return false;
  *tb_out = tb;
  grid[0] = g[0];
  grid[1] = g[1];
  grid128[0] = g128[0];
  grid128[1] = g128[1];
  return true;
}

}  // namespace ehc
