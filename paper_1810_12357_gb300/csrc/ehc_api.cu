// ehc_api.cu -- the C ABI of libehc (declared in include/ehc.h): argument
// checks, unit conversion, device memory, per-MD-step scalars, substep loops
// replayed from CUDA graphs, and the FP64 energy ledger.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ehc_internal.cuh"

// an NVTX range over one library call (named in profiler timelines; next to free
// when no tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

using namespace ehc;


struct ehc_ctx {
  Ctx c;
};

namespace {

// CODATA 2018
constexpr double kKB_EV = 8.617333262e-5;
constexpr double kKB_J = 1.380649e-23;
constexpr double kEV_J = 1.602176634e-19;
constexpr double kPI = 3.14159265358979323846;

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return EHC_E_CUDA;     \
  } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count) {
  return cudaMalloc((void **)p, sizeof(T) * (count > 0 ? count : 1));
}

int err_code(int32_t bits) {
  if (bits & ERR_INDEX) return EHC_E_INDEX;
  if (bits & ERR_BOUNDS) return EHC_E_BOUNDS;
  if (bits & ERR_NBR_OVERFLOW) return EHC_E_NBR_OVERFLOW;
  if (bits & (ERR_RANGE | ERR_SPEED)) return EHC_E_RANGE;
  if (bits & ERR_TIMEOUT) return EHC_E_TIMEOUT;
  return EHC_OK;
}

void free_all(Ctx &c) {
  cudaStream_t st = c.stream;
  cudaStreamSynchronize(st);
  void *dev[] = {c.type_orig, c.type_s, c.q_orig, c.cell_count, c.cell_start, c.cell_fill, c.scan_tmp,
                 c.perm, c.inv_perm[0], c.inv_perm[1], c.q_s, c.v_s, c.nbr, c.cnt, c.T[0], c.T[1],
                 c.dmir[0], c.dmir[1], c.abuf[0], c.abuf[1], c.Tl_f, c.Tl_d, c.depth_orig, c.srcw,
                 c.pulse, c.dKE, c.partials, c.scal, c.err, c.coef, c.x_dev, c.v_dev, c.T_out,
                 c.pidx, c.row_nbr, c.dlo, c.uTl, c.pulse_f, c.rrange[0], c.rrange[1], c.srcw_d, c.reps,
                 c.work, c.wgt, c.tfix_orig, c.bmask, c.bres, c.bnd_part, c.uhi, c.md_part, c.ldmax,
                 c.cand, c.ccnt, c.q_ref, c.perm_raw, c.wgt_d, c.rng_id};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (c.pulse_host) cudaFreeHost(c.pulse_host);
  if (c.scal_host) cudaFreeHost(c.scal_host);
  if (c.coef_host) cudaFreeHost(c.coef_host);
  if (c.pulse_f_host) cudaFreeHost(c.pulse_f_host);
  for (int i = 0; i < c.n_graphs; ++i) cudaGraphExecDestroy(c.graphs[i].exec);
  c.n_graphs = 0;
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  if (c.pulse_ev) cudaEventDestroy(c.pulse_ev);
  if (c.io_stream) cudaStreamDestroy(c.io_stream);
  for (cudaEvent_t e : c.io_ev)
    if (e) cudaEventDestroy(e);
}

// read back scal[0..15] and the error word; synchronises the stream
int readback(Ctx &c) {
  CK(cudaMemcpyAsync(c.scal_host, c.scal, sizeof(double) * 16, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(c.scal_host + 16, c.err, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  int32_t w[4];
  std::memcpy(w, c.scal_host + 16, sizeof(w));
  c.dev_err = w[0];
  return EHC_OK;
}

// neighbour rows of every row (cy, cz): z offset outer, y offset inner, wrapped on
// periodic axes, dropped outside non-periodic ones, duplicates removed, -1 padded
void row_table(const Grid &g, std::vector<int32_t> &tab) {
  const int64_t ny = g.nc[1], nz = g.nc[2];
  tab.assign((size_t)(ny * nz * kRowNbr), -1);
  for (int64_t cz = 0; cz < nz; ++cz)
    for (int64_t cy = 0; cy < ny; ++cy) {
      const int64_t R = cy + ny * cz;
      int m = 0;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
          int64_t z = cz + dz, y = cy + dy;
          if (g.per[2]) z = (z + nz) % nz;
          else if (z < 0 || z >= nz) continue;
          if (g.per[1]) y = (y + ny) % ny;
          else if (y < 0 || y >= ny) continue;
          const int32_t R2 = (int32_t)(y + ny * z);
          bool dup = false;
          for (int q = 0; q < m; ++q) dup |= tab[R * kRowNbr + q] == R2;
          if (!dup) tab[R * kRowNbr + m++] = R2;
        }
    }
}

double cap_SI(const Ctx &c) {
  return c.p.Ce_cap_kB > 0 ? c.p.Ce_cap_kB * kKB_J / (c.vatom * 1e-30) : 0.0;
}

// n_sub substeps on the context stream.  The single-precision path splits T
// into the float-float state first and merges it back at the end.  Loops of 4 or
// more substeps are captured once into a CUDA graph and replayed; the key holds
// everything a launch bakes in (buffer choice, path, pairs per atom).
cudaError_t enqueue_substeps(Ctx &c, int32_t n_sub, int p0, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < n_sub && e == cudaSuccess; ++k) e = launch_substep(c, k, p0 ^ (k & 1), st);
  return e;
}

// The single-precision path keeps its float-float state between substep calls;
// T (FP64) is rebuilt from it only when something reads T, and the state is
// split from T again only after something changed T.
int ensure_t(Ctx &c) {
  if (c.t_stale) {
    CK(launch_merge(c, c.parity, c.stream));
    c.t_stale = false;
    c.t_version += 1;
  }
  return EHC_OK;
}

int ensure_split(Ctx &c) {
  if (c.p.flux_prec == 0 && !c.ff_valid) {
    CK(launch_split(c, c.stream));
    // row value ranges of this snapshot are unknown: the first substep takes the
    // general polynomial everywhere
    if (c.nrows > 0) {
      CK(cudaMemsetAsync(c.rrange[c.parity], 0xfe, sizeof(float) * c.nrows, c.stream));
      CK(cudaMemsetAsync(c.rrange[c.parity] + c.nrows, 0x7f, sizeof(float) * c.nrows, c.stream));
    }
    c.ff_valid = true;
  }
  return EHC_OK;
}

int run_substeps(Ctx &c, int32_t n_sub) {
  c.t_version += 1;
  const int p0 = (c.p.flux_prec == 1) ? c.tcur : c.parity;
  const int ab = (c.A == c.abuf[0]) ? 0 : 1;
  const int path = (c.p.flux_prec == 1) ? 2 : ((tile_path(c) || local_tile(c)) ? 1 : 0);
  const int pairs = (c.n_max + 1) / 2;
  const int tile = c.tile_floats, nt = c.tile_nt * 8 + c.tile_q;   // width and grid share, both baked in
  const int border = c.has_border ? 1 : 0;
  bool use_graph = c.p.use_graph && n_sub >= 4;
  if (use_graph) {
    int hit = -1;
    for (int i = 0; i < c.n_graphs; ++i) {
      const auto &e = c.graphs[i];
      if (e.n_sub == n_sub && e.parity == p0 && e.tcur == c.tcur && e.abuf == ab && e.path == path &&
          e.pairs == pairs && e.tile == tile && e.nt == nt && e.border == border)
        hit = i;
    }
    if (hit < 0) {
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t le = enqueue_substeps(c, n_sub, p0, c.cap_stream);
      cudaError_t ee = cudaStreamEndCapture(c.cap_stream, &graph);
      if (le != cudaSuccess || ee != cudaSuccess) return EHC_E_CUDA;
      cudaGraphExec_t exec;
      cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) return EHC_E_CUDA;
      if (c.n_graphs == 8) {
        int lru = 0;
        for (int i = 1; i < 8; ++i)
          if (c.graphs[i].last_use < c.graphs[lru].last_use) lru = i;
        cudaGraphExecDestroy(c.graphs[lru].exec);
        c.graphs[lru] = c.graphs[7];
        c.n_graphs = 7;
      }
      c.graphs[c.n_graphs] = {n_sub, p0, c.tcur, ab, path, pairs, tile, nt, border, exec, 0};
      hit = c.n_graphs++;
    }
    c.graphs[hit].last_use = ++c.use_clock;
    CK(cudaGraphLaunch(c.graphs[hit].exec, c.stream));
  } else {
    CK(enqueue_substeps(c, n_sub, p0, c.stream));
  }
  const int p1 = p0 ^ (n_sub & 1);
  if (c.p.flux_prec == 1) {
    c.tcur = p1;
  } else {
    c.parity = p1;
    c.t_stale = true;
  }
  return EHC_OK;
}

// the row-tile kernel's arguments of one system
RepArgs rep_args(const Ctx &c);

// refresh the device argument table of the row-tile kernel (P changes per build)
cudaError_t upload_reps(Ctx &c) {
  const RepArgs ra = rep_args(c);
  return cudaMemcpy(c.reps, &ra, sizeof(ra), cudaMemcpyHostToDevice);
}

RepArgs rep_args(const Ctx &c) {
  RepArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  ra.n = (int32_t)c.n;
  ra.ncx = c.g.nc[0];
  int32_t P = (c.n_max + 1) / 2;
  if (P > (c.W + 1) / 2) P = (c.W + 1) / 2;
  ra.P = P;
  ra.nrows = (int32_t)c.nrows;
  ra.ps = (int32_t)c.ps;
  ra.start = c.cell_start;
  ra.row_nbr = c.row_nbr;
  ra.pidx = c.pidx;
  ra.dmir[0] = c.dmir[0];
  ra.dmir[1] = c.dmir[1];
  ra.lo = c.dlo;
  ra.A = c.A;
  ra.uTl = c.uTl;
  ra.srcw = c.srcw;
  ra.pulse_f = c.pulse_f;
  ra.fix = c.has_border ? c.bmask : nullptr;
  ra.res = c.bres;
  ra.uhi = c.uhi;
  ra.ldmax = c.ldmax;
  ra.rrange[0] = c.rrange[0];
  ra.rrange[1] = c.rrange[1];
  ra.cf = c.coef;
  ra.err = c.err;
  return ra;
}

}  // namespace

extern "C" {

const char *ehc_strerror(int code) {
  switch (code) {
    case EHC_OK: return "ok";
    case EHC_E_INVAL: return "invalid argument";
    case EHC_E_NOMEM: return "out of memory";
    case EHC_E_CUDA: return "CUDA runtime error";
    case EHC_E_UNSTABLE: return "substep unstable: dt (2 n_max K + G/C_e) > 2";
    case EHC_E_RANGE: return "normalised temperature left [0,1] (raise Tmax) or became NaN";
    case EHC_E_NBR_OVERFLOW: return "neighbour count exceeds max_neighbors";
    case EHC_E_TIMEOUT: return "bounded device wait timed out";
    case EHC_E_STATE: return "call out of order";
    case EHC_E_BOUNDS: return "atom outside a non-periodic box extent";
    case EHC_E_INDEX: return "gathered index outside its table (bounds-checked build)";
    default: return "unknown error";
  }
}

int ehc_create(const ehc_params *p, int64_t n_atoms, const double box_A[3], const int32_t periodic[3],
               const double *mass_amu_host, int32_t n_types, const int32_t *type_dev, void *stream,
               ehc_ctx **out) {
  if (!p || !box_A || !periodic || !mass_amu_host || !out) return EHC_E_INVAL;
  *out = nullptr;
  if (n_atoms < 0 || n_atoms >= (int64_t)INT32_MAX / 2) return EHC_E_INVAL;
  if (n_types < 1 || n_types > kMaxTypes || (n_types > 1 && !type_dev)) return EHC_E_INVAL;
  if (!(p->rc_A > 0) || !(p->dt_sub_fs > 0) || !(p->Tmax_K > 0) || !(p->zb2_A2 > 0) || p->dim_d < 1 ||
      !(p->gamma_Ce > 0) || !(p->kappa0 >= 0) || !(p->G >= 0) || p->Tref_K < 0 || p->Tref_K > p->Tmax_K)
    return EHC_E_INVAL;
  if (p->flux_prec != 0 && p->flux_prec != 1) return EHC_E_INVAL;
  if (p->couple_mode != 0 && p->couple_mode != 1) return EHC_E_INVAL;
  if (p->laser_on && (!(p->laser_lp_A > 0) || !(p->laser_sigma_fs > 0))) return EHC_E_INVAL;
  if (p->rate_shell_n < 0) return EHC_E_INVAL;
  if (p->ce_mode != 0 && p->ce_mode != 1) return EHC_E_INVAL;
  if (!(p->pot_D_eV >= 0) || (p->pot_D_eV > 0 && (!(p->pot_alpha_perA > 0) || !(p->pot_r0_A > 0))) ||
      !(p->stop_beta_per_fs >= 0) || !(p->stop_ecut_eV >= 0))
    return EHC_E_INVAL;
  int32_t W = p->max_neighbors <= 0 ? 32 : p->max_neighbors;
  if (W > kMaxWidth || W > 255) return EHC_E_INVAL;
  for (int t = 0; t < n_types; ++t)
    if (!(mass_amu_host[t] > 0)) return EHC_E_INVAL;

  ehc_ctx *h = new (std::nothrow) ehc_ctx();
  if (!h) return EHC_E_NOMEM;
  Ctx &c = h->c;
  c.p = *p;
  c.n = n_atoms;
  if (p->tile_threads != 0 && p->tile_threads != 128 && p->tile_threads != 256) {
    delete h;
    return EHC_E_INVAL;
  }
  c.tile_nt_fixed = p->tile_threads;
  if (p->tile_grid_quarters < 0 || p->tile_grid_quarters > 4 || (p->tile_grid_quarters && !p->tile_threads)) {
    delete h;
    return EHC_E_INVAL;
  }
  c.tile_q_fixed = p->tile_grid_quarters;
  c.W = W;
  c.stream = (cudaStream_t)stream;
  c.g.rcq = llrint(p->rc_A * 1048576.0);
  // cells at least r_c + |skin| wide (a negative skin: the same cells, full search every build)
  const double skin = p->skin_A;
  if (!(skin == skin) || std::fabs(skin) > p->rc_A) { delete h; return EHC_E_INVAL; }
  const int64_t cellq = llrint((p->rc_A + std::fabs(skin)) * 1048576.0);
  c.skin_q = skin > 0 ? cellq - c.g.rcq : 0;
  int64_t ncell = 1;
  for (int k = 0; k < 3; ++k) {
    c.box[k] = box_A[k];
    if (!(box_A[k] > 0)) { delete h; return EHC_E_INVAL; }
    c.g.Lq[k] = llrint(box_A[k] * 1048576.0);
    if (c.g.Lq[k] <= 0 || c.g.Lq[k] >= INT32_MAX) { delete h; return EHC_E_INVAL; }
    c.g.per[k] = periodic[k] ? 1 : 0;
    if (c.g.per[k] && c.g.Lq[k] <= 2 * c.g.rcq) { delete h; return EHC_E_INVAL; }
    // the candidate radius must keep a unique minimum image too
    if (c.g.per[k] && c.g.Lq[k] <= 2 * cellq) c.skin_q = 0;
    int64_t nc = c.g.Lq[k] / cellq;
    if (nc < 1) nc = 1;
    if (nc > 1024) nc = 1024;
    c.g.nc[k] = (int32_t)nc;
    ncell *= nc;
  }
  // very large, sparse boxes: coarser cells (still at least r_c wide) keep the cell arrays bounded
  while (ncell > (int64_t(1) << 26)) {
    int k = 0;
    for (int j = 1; j < 3; ++j)
      if (c.g.nc[j] > c.g.nc[k]) k = j;
    ncell /= c.g.nc[k];
    c.g.nc[k] = (c.g.nc[k] + 1) / 2;
    ncell *= c.g.nc[k];
  }
  c.g.ncell = ncell;
  c.mt.n_types = n_types;
  for (int t = 0; t < kMaxTypes; ++t) c.mt.m[t] = t < n_types ? mass_amu_host[t] : mass_amu_host[0];
  c.vatom = p->vatom_A3 > 0 ? p->vatom_A3 : (n_atoms > 0 ? box_A[0] * box_A[1] * box_A[2] / (double)n_atoms : 1.0);
  c.cap_si = cap_SI(c);
  c.local = p->ce_mode == 1;
  c.max_sub = 65536;

  const int64_t n = n_atoms;
  const int64_t ntiles = (ncell + 4095) / 4096;
  bool ok = true;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  if (n_types > 1) A(dalloc(&c.type_orig, n));
  A(dalloc(&c.type_s, n));
  A(dalloc(&c.q_orig, n));
  A(dalloc(&c.cell_count, ncell + 1));
  A(dalloc(&c.cell_start, ncell + 1));
  A(dalloc(&c.cell_fill, ncell));
  A(dalloc(&c.scan_tmp, ntiles + 1));
  A(dalloc(&c.perm, n));
  A(dalloc(&c.perm_raw, n));
  A(dalloc(&c.inv_perm[0], n));
  A(dalloc(&c.inv_perm[1], n));
  A(dalloc(&c.q_s, n));
  A(dalloc(&c.v_s, n));
  A(dalloc(&c.nbr, (size_t)W * n));
  if (c.p.rate_shell_n > 0) A(dalloc(&c.wgt, (size_t)W * n));
  if (c.p.rate_shell_n > 0 && c.p.flux_prec == 1) A(dalloc(&c.wgt_d, (size_t)W * n));
  c.ps = (n + 3) / 4 * 4;
  A(dalloc(&c.pidx, (size_t)((W + 1) / 2) * (size_t)(c.ps > 0 ? c.ps : 4)));
  A(dalloc(&c.dlo, n));
  if (c.local) A(dalloc(&c.uhi, n));
  if (c.local) A(dalloc(&c.ldmax, 3));
  A(dalloc(&c.uTl, n));
  A(dalloc(&c.pulse_f, c.max_sub));
  c.nrows = (int64_t)c.g.nc[1] * c.g.nc[2];
  A(dalloc(&c.row_nbr, c.nrows * kRowNbr));
  A(dalloc(&c.cnt, n));
  A(dalloc(&c.T[0], n));
  A(dalloc(&c.T[1], n));
  A(dalloc(&c.dmir[0], c.ps > 0 ? c.ps : 4));   // padded: tiles are copied in 16-byte aligned supersets
  A(dalloc(&c.dmir[1], c.ps > 0 ? c.ps : 4));
  A(dalloc(&c.abuf[0], n));
  A(dalloc(&c.abuf[1], n));
  A(dalloc(&c.Tl_f, n));
  A(dalloc(&c.Tl_d, n));
  A(dalloc(&c.depth_orig, n));
  A(dalloc(&c.srcw, n));
  A(dalloc(&c.srcw_d, n));
  A(dalloc(&c.pulse, c.max_sub));
  A(dalloc(&c.dKE, n));
  A(dalloc(&c.partials, kRedBlocks * 6));
  A(dalloc(&c.md_part, md_force_blocks(n)));
  // device scalars, one slot per use (host mirror: scal_host[0..15], error words at [16..17]):
  //   0-5 system sums of the build and the ledger (sum T, max T / sum U, sum KE, ...),
  //   6-7 ehc_sums_at, 8 E_lat, 9 stopped-atom count (u64 bits), 10-11 border reservoirs,
  //   12 ehc_probe_wait flag (int32), 13 ehc_max_speed result, 14 ehc_forces potential energy
  A(dalloc(&c.scal, 16));
  A(dalloc(&c.err, 8));
  if (c.skin_q > 0) {
    A(dalloc(&c.cand, (int64_t)kCandWidth * (n > 0 ? n : 1)));
    A(dalloc(&c.ccnt, n > 0 ? n : 1));
    A(dalloc(&c.q_ref, n > 0 ? n : 1));
  }
  A(dalloc(&c.coef, 1));
  A(dalloc(&c.x_dev, 3 * n));
  A(dalloc(&c.v_dev, 3 * n));
  A(dalloc(&c.T_out, n));
  A(cudaMallocHost((void **)&c.pulse_host, sizeof(double) * c.max_sub));
  A(cudaMallocHost((void **)&c.scal_host, sizeof(double) * 24));
  A(cudaMallocHost((void **)&c.coef_host, sizeof(StepCoef)));
  A(cudaMallocHost((void **)&c.pulse_f_host, sizeof(float) * c.max_sub));
  A(dalloc(&c.rrange[0], 2 * c.nrows));
  A(dalloc(&c.rrange[1], 2 * c.nrows));
  A(dalloc(&c.reps, 1));
  A(dalloc(&c.work, c.nrows));
  A(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, 0));
  A(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
  A(cudaEventCreateWithFlags(&c.pulse_ev, cudaEventDisableTiming));
  A(cudaStreamCreateWithFlags(&c.io_stream, cudaStreamNonBlocking));
  for (cudaEvent_t &e : c.io_ev) A(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  if (!ok) {
    cudaGetLastError();
    free_all(c);
    delete h;
    return EHC_E_NOMEM;
  }
  c.A = c.abuf[0];
  c.A_tmp = c.abuf[1];
  c.maxcnt = c.err + 1;
  c.maxstaged = c.err + 2;
  c.maxrow = c.err + 3;
  std::vector<int32_t> rt;
  row_table(c.g, rt);
  cudaError_t e = cudaSuccess;
  if (n_types > 1 && n > 0)
    e = cudaMemcpyAsync(c.type_orig, type_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.scal, 0, sizeof(double) * 16, c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.err, 0, sizeof(int32_t) * 8, c.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c.row_nbr, rt.data(), sizeof(int32_t) * rt.size(), cudaMemcpyHostToDevice, c.stream);
  std::vector<int2> wl((size_t)c.nrows);
  for (int64_t R = 0; R < c.nrows; ++R) wl[(size_t)R] = make_int2(0, (int)R);
  c.nwork = (int32_t)c.nrows;
  if (e == cudaSuccess && c.nrows > 0)
    e = cudaMemcpyAsync(c.work, wl.data(), sizeof(int2) * wl.size(), cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = upload_reps(c);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.abuf[0], 0, sizeof(double) * (n > 0 ? n : 1), c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.srcw, 0, sizeof(float) * (n > 0 ? n : 1), c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    free_all(c);
    delete h;
    return EHC_E_CUDA;
  }
  *out = h;
  return EHC_OK;
}

void ehc_destroy(ehc_ctx *h) {
  if (!h) return;
  free_all(h->c);
  delete h;
}

int ehc_set_te(ehc_ctx *h, const double *Te_dev) {
  NvtxRange nvtx_range("ehc_set_te");
  if (!h || (!Te_dev && h->c.n > 0)) return EHC_E_INVAL;
  Ctx &c = h->c;
  c.t_version += 1;
  if (c.n > 0) {
    CK(cudaMemcpyAsync(c.T[c.tcur], Te_dev, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
    CK(cudaMemsetAsync(c.A, 0, sizeof(double) * c.n, c.stream));
  }
  CK(cudaMemsetAsync(c.scal, 0, sizeof(double) * 16, c.stream));
  CK(launch_seed(c, cap_SI(c)));
  int r = readback(c);
  if (r) return r;
  c.te_orig_order = true;
  c.have_te = true;
  c.built = false;
  c.ff_valid = false;
  c.t_stale = false;
  c.E_e0 = c.scal_host[2] * c.vatom * 1e-30 / kEV_J;
  c.E_base = c.E_e0;
  c.ST_base = c.scal_host[0];
  c.VC_prev = -1;
  c.E_src = 0;
  c.E_res = 0;
  c.md_step = 0;
  return EHC_OK;
}

int ehc_set_border(ehc_ctx *h, const double *Tfix_dev) {
  if (!h) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (c.local && Tfix_dev) return EHC_E_STATE;   // the border is a form of the global C_e only
  if (!Tfix_dev || c.n == 0) {
    c.border_next = false;
    return EHC_OK;
  }
  if (!c.tfix_orig) {
    const int64_t n = c.n;
    bool ok = true;
    auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
    A(dalloc(&c.tfix_orig, n));
    A(dalloc(&c.bmask, n));
    A(dalloc(&c.bres, n));
    A(dalloc(&c.bnd_part, (int64_t)border_red_blocks()));
    if (ok) A(cudaMemsetAsync(c.bres, 0, sizeof(double) * n, c.stream));
    if (!ok) {
      cudaGetLastError();
      for (void **q : {(void **)&c.tfix_orig, (void **)&c.bmask, (void **)&c.bres, (void **)&c.bnd_part}) {
        if (*q) cudaFree(*q);
        *q = nullptr;
      }
      return EHC_E_NOMEM;
    }
  }
  CK(cudaMemcpyAsync(c.tfix_orig, Tfix_dev, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
  c.border_next = true;
  return EHC_OK;
}

int ehc_set_depth(ehc_ctx *h, const double *depth_dev) {
  if (!h || (!depth_dev && h->c.n > 0)) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (c.n > 0)
    CK(cudaMemcpyAsync(c.depth_orig, depth_dev, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
  c.have_depth = true;
  return EHC_OK;
}

}  // extern "C"

namespace {

// first half of a neighbour build: queue every kernel and the copies of the
// per-step scalars to pinned host memory (no synchronisation)
// v_ready (if not null): an event after which v_dev holds the velocities; the
// stream waits for it only before the velocity gather, after the neighbour search
int build_enqueue(Ctx &c, const double *x_dev, const double *v_dev, cudaEvent_t v_ready = nullptr) {
  c.t_version += 1;
  if (!c.have_te) return EHC_E_STATE;
  if (c.n > 0 && (!x_dev || !v_dev)) return EHC_E_INVAL;
  int r0 = ensure_t(c);
  if (r0) return r0;
  c.ff_valid = false;
  // the reservoirs of the closing MD step into scal[10], cleared, before the re-sort
  if (c.bres) CK(border_flush(c, c.scal + 10, true));
  CK(launch_bin(c, x_dev));
  CK(launch_sort_cells(c));
  // with velocities still in flight the gather leaves them to a second pass after
  // the neighbour search
  CK(launch_gather(c, v_ready ? nullptr : v_dev, c.te_orig_order));
  c.te_orig_order = false;
  c.has_border = c.border_next;
  CK(launch_neighbors(c));
  if (v_ready) {
    CK(cudaStreamWaitEvent(c.stream, v_ready, 0));
    CK(launch_gather_vel(c, v_dev));
  }
  CK(launch_lattice_temperature(c));
  CK(launch_globals(c));
  // border of the new sort order: after the means, so that the closing step's
  // ledger sees the temperatures before border atoms are set to T_b
  if (c.has_border) CK(border_apply(c));
  CK(cudaMemcpyAsync(c.scal_host, c.scal, sizeof(double) * 16, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(c.scal_host + 16, c.err, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, c.stream));
  return EHC_OK;
}

// per-step scalars from the system means of the step (Sec. 2: mean electronic
// temperature, classical lattice temperature): C_e, kappa_e, K of Eq. Kij, the
// stability number and the coefficient upload
int step_coefficients(Ctx &c, double Te_mean, double Tlat) {
  c.Te_mean = Te_mean;
  c.Tlat = Tlat;
  double Ce = c.p.gamma_Ce * c.Te_mean;
  const double cap = cap_SI(c);
  if (cap > 0 && Ce > cap) Ce = cap;
  if (c.n == 0) Ce = c.p.gamma_Ce;   // nothing to advance; keep the coefficients finite
  if (!(Ce > 0)) return EHC_E_RANGE;
  double kappa = c.p.kappa0;
  if (c.p.kappa_mode == 1) kappa = c.Tlat > 0 ? c.p.kappa0 * c.Te_mean / c.Tlat : c.p.kappa0;
  c.Ce = Ce;
  // Eq. Kij, K = 2 kappa_e d / (C_e Z b^2): m^2/s over A^2 -> 1/fs
  c.K = 2.0 * c.p.dim_d * kappa / (Ce * c.p.zb2_A2 * 1e-20) * 1e-15;
  c.cG = c.p.G / Ce * 1e-15;
  c.VG = c.p.G * c.vatom * 1e-30 / kEV_J * 1e-15;
  c.VC = c.vatom * 1e-30 * Ce / kEV_J;
  c.gammaL = c.p.G * c.vatom * 1e-30 / (3.0 * kKB_J) * 1e-15;
  c.stability = c.p.dt_sub_fs * (2.0 * c.n_max * c.K + c.cG);
  c.VC_prev = c.VC;
  if (c.local) {
    // LOCAL form: pair energy rates (2 d / Z b^2) kappa_ij Tmax f_ij, kappa_ij the
    // mean of kappa0 T / T_lat (or kappa0) of the two atoms, in units of gamma Tmax^2
    const double gam = c.p.gamma_Ce, Tm = c.p.Tmax_K;
    const double geo = 2.0 * c.p.dim_d / (c.p.zb2_A2 * 1e-20);
    const double dts = c.p.dt_sub_fs * 1e-15;
    double Ku;   // [1/s]
    if (c.p.kappa_mode == 1) Ku = c.Tlat > 0 ? geo * c.p.kappa0 / (gam * c.Tlat) : HUGE_VAL;
    else Ku = geo * c.p.kappa0 / (gam * Tm);
    c.K = Ku * 1e-15;
    // stability: dt (2 n_max K_hi + G / C_min) with the rate of the energy
    // variables: kappa_mode 1, Ku (times T_hi / T_c above the cap); mode 0,
    // 2 d kappa0 / (Z b^2 C_e(T_min))
    const double cap = c.cap_si;
    auto ce = [&](double T) { return (cap > 0 && gam * T > cap) ? cap : gam * T; };
    const double Tc = cap > 0 ? cap / gam : HUGE_VAL;
    const double Thi = c.scal_host[1];
    double Khi;
    if (c.p.kappa_mode == 1) Khi = Ku * (Thi > Tc ? Thi / Tc : 1.0);
    else Khi = c.Tmin > 0 ? geo * c.p.kappa0 / ce(c.Tmin) : HUGE_VAL;
    const double cmin = ce(c.Tmin);
    c.cG = (cmin > 0 ? c.p.G / cmin : HUGE_VAL) * 1e-15;
    c.stability = c.p.dt_sub_fs * (2.0 * c.n_max * Khi * 1e-15 + c.cG);
  }
  StepCoef &cf = *c.coef_host;
  cf.dt = c.p.dt_sub_fs;
  cf.dtTK = c.p.dt_sub_fs * c.p.Tmax_K * c.K;
  cf.dtcG = c.p.dt_sub_fs * c.cG;
  cf.dtVG = c.p.dt_sub_fs * c.VG;
  cf.invTmax = 1.0 / c.p.Tmax_K;
  cf.Tref = c.p.Tref_K;
  cf.th_ref = (float)(c.p.Tref_K / c.p.Tmax_K);
  cf.omt = (float)(1.0 - c.p.Tref_K / c.p.Tmax_K);
  cf.dtK_f = (float)(c.p.dt_sub_fs * c.K);
  cf.dtcGn_f = (float)(c.p.dt_sub_fs * c.cG / c.p.Tmax_K);
  cf.Tmax_f = (float)c.p.Tmax_K;
  cf.pad[0] = cf.pad[1] = cf.pad[2] = 0.f;
  {
    const double gam = c.p.gamma_Ce, Tm = c.p.Tmax_K;
    const double th = c.p.Tref_K / Tm;
    const double thc = c.cap_si > 0 ? c.cap_si / gam / Tm : 0.0;
    auto u = [&](double t) { return (thc > 0 && t > thc) ? thc * t - 0.5 * thc * thc : 0.5 * t * t; };
    cf.dtKu = c.local ? c.p.dt_sub_fs * c.K : 0.0;
    cf.dtgu = c.p.dt_sub_fs * 1e-15 * c.p.G / (gam * Tm * Tm);
    cf.thc = thc;
    cf.u_ref = u(th);
    cf.dtKu_f = (float)cf.dtKu;
    cf.dtgu_f = (float)cf.dtgu;
    cf.thc_f = (float)thc;
    cf.inv_thc_f = thc > 0 ? (float)(1.0 / thc) : 0.f;
    cf.wc_f = thc > 0 ? (float)(0.5 * thc * thc - cf.u_ref) : 0.f;
    cf.thsq_f = (float)(th * th);
    cf.kmode = c.p.kappa_mode == 1 ? 1 : 0;
    cf.pad2 = 0.f;
    cf.dtVGu = (double)cf.dtgu_f * c.vatom * 1e-30 * gam * Tm * Tm / kEV_J;
  }
  CK(cudaMemcpyAsync(c.coef, c.coef_host, sizeof(StepCoef), cudaMemcpyHostToDevice, c.stream));
  return EHC_OK;
}

// second half, after the stream has been synchronised: per-step scalars (Sec. 2
// means, C_e, kappa_e, Eq. Kij), ledger, stability, coefficient upload
int build_finish(Ctx &c, bool own_tiles) {
  int32_t w[4];
  std::memcpy(w, c.scal_host + 16, sizeof(w));
  c.dev_err = w[0];
  c.n_max = w[1];
  c.staged_max = w[2];
  c.row_max = w[3];
  c.builds += 1;
  // size the row-tile buffers (grown only when a build outgrows them)
  if (own_tiles && c.p.flux_prec == 0 && c.staged_max > c.tile_floats) {
    int32_t tb = 0, grid[2] = {0, 0}, grid128[2] = {0, 0};
    if (tile_size(c.staged_max, c.num_sms, &tb, grid, grid128)) {
      c.tile_floats = tb;
      c.tile_nt = 0;
      c.tile_grid128[0] = grid128[0];
      c.tile_grid128[1] = grid128[1];
      c.tile_grid[0] = grid[0];
      c.tile_grid[1] = grid[1];
    }
  }
  const double sumT = c.scal_host[0], sumKE = c.scal_host[2];
  c.wsum = c.scal_host[3];
  c.Tmin = -c.scal_host[4];
  // ledger: close the previous MD step with its own C_e (the LOCAL form's E_e is
  // evaluated directly from the temperatures)
  if (c.VC_prev > 0 && !c.local) {
    c.E_base += c.VC_prev * (sumT - c.ST_base);
    c.ST_base = sumT;
    if (c.bres) c.E_res += c.VC_prev * c.scal_host[10] * (c.p.flux_prec == 1 ? 1.0 : c.p.Tmax_K);
  }
  // system means (Sec. 2): mean electronic temperature, classical T_lat = K / ((3/2) k_B N)
  const double N = (double)(c.n > 0 ? c.n : 1);
  const int rc = step_coefficients(c, sumT / N, sumKE / (1.5 * kKB_EV * N));
  if (rc) return rc;
  if (own_tiles) CK(upload_reps(c));   // a batch keeps its own table of every replica
  c.built = true;
  return err_code(c.dev_err);
}

}  // namespace

extern "C" {

int ehc_build_neighbors(ehc_ctx *h, const double *x_dev, const double *v_dev) {
  NvtxRange nvtx_range("ehc_build_neighbors");
  if (!h) return EHC_E_INVAL;
  Ctx &c = h->c;
  int r = build_enqueue(c, x_dev, v_dev);
  if (r) return r;
  CK(cudaStreamSynchronize(c.stream));
  return build_finish(c, true);
}


}  // extern "C"

namespace {

// Tuner of the row-tile kernel: the widths (256, 128 threads owning atoms) and
// the persistent grid's share of the resident CTAs (4, 3, 2 quarters), timed with
// events on the stream over two substeps each, twelve in all (an even count per
// candidate, so the mirror parity is unchanged).  Another choice must beat the
// first (256, full grid) by 3 %.  Every choice gives the same results: each
// atom's arithmetic does not depend on the schedule.
constexpr int kTuneCands = 6;
template <typename Launch>
int tune_tiles(cudaStream_t st, int32_t *nt_out, int32_t *q_out, Launch launch) {
  const int32_t nts[kTuneCands] = {256, 256, 256, 128, 128, 128};
  const int32_t qs[kTuneCands] = {4, 3, 2, 4, 3, 2};
  cudaEvent_t ev[kTuneCands + 1];
  for (int i = 0; i <= kTuneCands; ++i) CK(cudaEventCreate(&ev[i]));
  CK(cudaEventRecord(ev[0], st));
  for (int i = 0; i < kTuneCands; ++i) {
    for (int k = 0; k < 2; ++k) CK(launch(2 * i + k, nts[i], qs[i]));
    CK(cudaEventRecord(ev[i + 1], st));
  }
  CK(cudaEventSynchronize(ev[kTuneCands]));
  float best = 0.f;
  int bi = 0;
  for (int i = 0; i < kTuneCands; ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
    if (i == 0) best = t;
    else if (t < 0.97f * best) {
      best = t;
      bi = i;
    }
  }
  for (int i = 0; i <= kTuneCands; ++i) cudaEventDestroy(ev[i]);
  *nt_out = nts[bi];
  *q_out = qs[bi];
  return EHC_OK;
}

}  // namespace

extern "C" {

int ehc_substep(ehc_ctx *h, int32_t n_sub, double t_fs) {
  NvtxRange nvtx_range("ehc_substep");
  if (!h || n_sub < 0) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.built) return EHC_E_STATE;
  if (n_sub == 0 || c.n == 0) return EHC_OK;
  if (!(c.stability <= 2.0)) return EHC_E_UNSTABLE;
  const bool laser = c.p.laser_on && c.have_depth;
  int32_t done = 0;
  while (done < n_sub) {
    int32_t chunk = n_sub - done;
    if (laser && chunk > c.max_sub) chunk = c.max_sub;
    if (laser) {
      CK(cudaEventSynchronize(c.pulse_ev));  // previous copy out of the staging buffer finished
      const double sig = c.p.laser_sigma_fs;
      const double S0 = c.p.laser_fluence_Jm2 / (c.p.laser_lp_A * 1e-10) / (sig * 1e-15 * std::sqrt(2.0 * kPI));
      for (int k = 0; k < chunk; ++k) {
        const double t = t_fs + c.p.dt_sub_fs * (double)(done + k);
        const double u = (t - c.p.laser_t0_fs) / sig;
        if (c.local) {
          // LOCAL form: the source's energy density in units of gamma Tmax^2 per fs
          const double gT2 = c.p.gamma_Ce * c.p.Tmax_K * c.p.Tmax_K;
          const double rate = S0 * std::exp(-0.5 * u * u) / gT2 * 1e-15;
          c.pulse_host[k] = rate;
          const float cf = (float)(c.p.dt_sub_fs * rate);
          c.pulse_f_host[k] = cf;
          const double eV_per_u = c.vatom * 1e-30 * gT2 / kEV_J;
          if (c.p.flux_prec == 1) c.E_src += eV_per_u * c.p.dt_sub_fs * rate * c.wsum;
          else c.E_src += eV_per_u * (double)cf * c.wsum;
          continue;
        }
        const double rate = S0 * std::exp(-0.5 * u * u) / c.Ce * 1e-15;  // K / fs at depth 0
        c.pulse_host[k] = rate;
        // the single-precision path adds the exact product of these two floats per atom
        const float cf = (float)(c.p.dt_sub_fs * rate / c.p.Tmax_K);
        c.pulse_f_host[k] = cf;
        if (c.p.flux_prec == 1) c.E_src += c.VC * c.p.dt_sub_fs * rate * c.wsum;
        else c.E_src += c.VC * c.p.Tmax_K * (double)cf * c.wsum;
      }
      CK(cudaMemcpyAsync(c.pulse, c.pulse_host, sizeof(double) * chunk, cudaMemcpyHostToDevice, c.stream));
      CK(cudaMemcpyAsync(c.pulse_f, c.pulse_f_host, sizeof(float) * chunk, cudaMemcpyHostToDevice, c.stream));
      CK(cudaEventRecord(c.pulse_ev, c.stream));
    }
    int r = ensure_split(c);
    if (r) return r;
    int32_t rest = chunk;
    const int pw = ((c.n_max + 1) / 2 == 9) ? 0 : 1;
    if (c.tile_nt_fixed) {
      c.tile_nt = c.tile_nt_fixed;
      c.tile_q = c.tile_q_fixed ? c.tile_q_fixed : 4;
    }
    if (!laser && c.tile_nt == 0 && chunk >= 2 * kTuneCands + 4 && tile_path(c) && c.tile_grid128[pw] > 0) {
      const int p0 = c.parity;
      c.t_version += 1;
      int32_t chosen = 256, q = 4;
      r = tune_tiles(c.stream, &chosen, &q, [&](int k, int nt, int qq) {
        c.tile_nt = nt;
        c.tile_q = qq;
        return launch_substep(c, k, p0 ^ (k & 1), c.stream);
      });
      c.tile_nt = chosen;
      c.tile_q = q;
      if (r) return r;
      c.t_stale = true;
      rest -= 2 * kTuneCands;   // an even count: the mirror parity is unchanged
    }
    r = run_substeps(c, rest);
    if (r) return r;
    done += chunk;
  }
  return EHC_OK;
}

int ehc_couple(ehc_ctx *h, double *v_dev, double dt_md_fs) {
  NvtxRange nvtx_range("ehc_couple");
  if (!h) return EHC_E_INVAL;
  Ctx &c = h->c;
  c.t_version += 1;
  if (!c.built) return EHC_E_STATE;
  if (c.n > 0 && !v_dev && !c.p.frozen) return EHC_E_INVAL;
  int r = ensure_t(c);
  if (r) return r;
  CK(launch_couple(c, v_dev, dt_md_fs));
  c.ff_valid = false;
  c.md_step += 1;
  return EHC_OK;
}

int ehc_forces(ehc_ctx *h, double *F_dev, double *epot_host) {
  NvtxRange nvtx_range("ehc_forces");
  if (!h || (h->c.n > 0 && !F_dev)) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.built) return EHC_E_STATE;
  CK(launch_forces(c, F_dev, c.md_part, c.scal + 14));
  if (epot_host) {
    CK(cudaMemcpyAsync(c.scal_host + 14, c.scal + 14, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    *epot_host = c.scal_host[14];
  }
  return EHC_OK;
}

int ehc_kick(ehc_ctx *h, double *v_dev, const double *F_dev, double dt_fs) {
  if (!h || (h->c.n > 0 && (!v_dev || !F_dev)) || !(dt_fs == dt_fs)) return EHC_E_INVAL;
  CK(launch_kick(h->c, v_dev, F_dev, dt_fs));
  return EHC_OK;
}

int ehc_get_te_at(ehc_ctx *h, const int32_t *idx_dev, int64_t m, double *out_dev) {
  if (!h || m < 0 || (m > 0 && (!idx_dev || !out_dev))) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.have_te) return EHC_E_STATE;
  int r = ensure_t(c);
  if (r) return r;
  CK(launch_get_at(c, idx_dev, m, out_dev));
  return EHC_OK;
}

int ehc_set_te_at(ehc_ctx *h, const int32_t *idx_dev, int64_t m, const double *vals_dev) {
  if (!h || m < 0 || (m > 0 && (!idx_dev || !vals_dev))) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.have_te) return EHC_E_STATE;
  if (m == 0) return EHC_OK;
  c.t_version += 1;
  CK(launch_set_at(c, idx_dev, m, vals_dev));
  // the row tiles' value ranges no longer cover the new values: the next substep
  // takes the full series everywhere
  if (c.p.flux_prec == 0 && c.ff_valid && c.nrows > 0) {
    CK(cudaMemsetAsync(c.rrange[c.parity], 0xfe, sizeof(float) * c.nrows, c.stream));
    CK(cudaMemsetAsync(c.rrange[c.parity] + c.nrows, 0x7f, sizeof(float) * c.nrows, c.stream));
  }
  return EHC_OK;
}

int ehc_sums_at(ehc_ctx *h, const int32_t *idx_dev, int64_t m, double *sums_host) {
  if (!h || !sums_host || m < 0 || (m > 0 && !idx_dev)) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.built) return EHC_E_STATE;
  int r = ensure_t(c);
  if (r) return r;
  if (m == 0 || c.n == 0) {
    sums_host[0] = sums_host[1] = 0.0;
    return EHC_OK;
  }
  // block sums in the global reductions' buffer (kRedBlocks x 6 >= 2 x 152 doubles),
  // the result in scal[6..7]
  CK(launch_sums_at(c, idx_dev, m, c.partials, c.scal + 6));
  CK(cudaMemcpyAsync(c.scal_host + 6, c.scal + 6, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(c.scal_host + 16, c.err, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  sums_host[0] = c.scal_host[6];
  sums_host[1] = c.scal_host[7];
  int32_t w[4];
  std::memcpy(w, c.scal_host + 16, sizeof(w));
  return (w[0] & ERR_INDEX) ? EHC_E_INDEX : EHC_OK;
}

int ehc_set_step_means(ehc_ctx *h, double Te_mean, double Tlat) {
  if (!h || !(Te_mean >= 0) || !(Tlat >= 0)) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.built) return EHC_E_STATE;
  return step_coefficients(c, Te_mean, Tlat);
}

int ehc_set_rng_ids(ehc_ctx *h, const int64_t *ids_dev, int64_t md_step) {
  if (!h || md_step < 0) return EHC_E_INVAL;
  Ctx &c = h->c;
  c.md_step = md_step;
  if (!ids_dev) {
    if (c.rng_id) CK(cudaStreamSynchronize(c.stream));   // a hand-over in flight may still read it
    if (c.rng_id) cudaFree(c.rng_id);
    c.rng_id = nullptr;
    return EHC_OK;
  }
  if (!c.rng_id && c.n > 0 && cudaMalloc((void **)&c.rng_id, sizeof(int64_t) * (size_t)c.n) != cudaSuccess) {
    cudaGetLastError();
    c.rng_id = nullptr;
    return EHC_E_NOMEM;
  }
  if (c.n > 0)
    CK(cudaMemcpyAsync(c.rng_id, ids_dev, sizeof(int64_t) * (size_t)c.n, cudaMemcpyDeviceToDevice, c.stream));
  return EHC_OK;
}

int ehc_probe_wait(ehc_ctx *h, uint32_t polls, int32_t complete) {
  if (!h || polls == 0) return EHC_E_INVAL;
  Ctx &c = h->c;
  // its own word (scal[12] as int32): the context's sticky error word stays untouched
  int32_t *flag = reinterpret_cast<int32_t *>(c.scal + 12);
  CK(cudaMemsetAsync(flag, 0, sizeof(int32_t), c.stream));
  CK(launch_wait_probe(polls, complete ? 1 : 0, flag, c.stream));
  int32_t got = 0;
  CK(cudaMemcpyAsync(&c.scal_host[12], flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  std::memcpy(&got, &c.scal_host[12], sizeof(got));
  return (got & ERR_TIMEOUT) ? EHC_E_TIMEOUT : EHC_OK;
}

int ehc_max_speed(ehc_ctx *h, const double *v_dev, double *vmax_host) {
  if (!h || !vmax_host || (h->c.n > 0 && !v_dev)) return EHC_E_INVAL;
  Ctx &c = h->c;
  CK(launch_vmax(c, v_dev, c.partials, kRedBlocks, c.scal + 13));
  CK(cudaMemcpyAsync(c.scal_host + 13, c.scal + 13, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  *vmax_host = c.scal_host[13];
  return EHC_OK;
}

int ehc_drift(ehc_ctx *h, double *x_dev, const double *v_dev, double dt_fs) {
  NvtxRange nvtx_range("ehc_drift");
  if (!h || (h->c.n > 0 && (!x_dev || !v_dev))) return EHC_E_INVAL;
  CK(launch_drift(h->c, x_dev, v_dev, dt_fs));
  return EHC_OK;
}

int ehc_sync(ehc_ctx *h) {
  if (!h) return EHC_E_INVAL;
  Ctx &c = h->c;
  CK(cudaMemcpyAsync(c.scal_host + 16, c.err, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  int32_t w[4];
  std::memcpy(w, c.scal_host + 16, sizeof(w));
  c.dev_err = w[0];
  return err_code(c.dev_err);
}

int ehc_energy(ehc_ctx *h, ehc_energy_t *out) {
  NvtxRange nvtx_range("ehc_energy");
  if (!h || !out) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.have_te) return EHC_E_STATE;
  int r0 = ensure_t(c);
  if (r0) return r0;
  CK(launch_ledger(c));
  if (c.bres) CK(border_flush(c, c.scal + 11, false));
  int r = readback(c);
  if (r) return r;
  const double sumT = c.scal_host[0];
  std::memset(out, 0, sizeof(*out));
  out->E_e = c.E_base + (c.VC_prev > 0 ? c.VC_prev * (sumT - c.ST_base) : 0.0);
  if (c.local) out->E_e = c.scal_host[5] * c.vatom * 1e-30 / kEV_J;   // sum_i V_atom U(T_i)
  out->E_lat = c.scal_host[8];
  out->E_src = c.E_src;
  out->E_e0 = c.E_e0;
  // the border's reservoirs: closed MD steps, and the current one with its C_e
  out->E_res = c.E_res + (c.bres && c.VC_prev > 0
                               ? c.VC_prev * c.scal_host[11] * (c.p.flux_prec == 1 ? 1.0 : c.p.Tmax_K)
                               : 0.0);
  const double scale = std::max(std::fabs(c.E_e0), std::fabs(out->E_e));
  out->drift = scale > 0 ? (out->E_e + out->E_lat - out->E_src + out->E_res - out->E_e0) / scale : 0.0;
  out->sum_T = sumT;
  out->max_T = c.scal_host[1];
  out->mean_T = c.n > 0 ? sumT / (double)c.n : 0.0;
  out->Te_mean_step = c.Te_mean;
  out->Tlat_step = c.Tlat;
  out->Ce_SI = c.Ce;
  out->K_per_fs = c.K;
  out->stability = c.stability;
  uint64_t ns;
  std::memcpy(&ns, c.scal_host + 9, sizeof(ns));
  out->n_stopped = (int64_t)ns;
  out->md_step = c.md_step;
  out->max_count = c.n_max;
  out->device_error = c.dev_err;
  return err_code(c.dev_err);
}

int ehc_get_te(ehc_ctx *h, double *Te_dev_out) {
  if (!h || (!Te_dev_out && h->c.n > 0)) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.have_te) return EHC_E_STATE;
  int r = ensure_t(c);
  if (r) return r;
  CK(launch_unpermute(c, c.T[c.tcur], Te_dev_out, c.te_orig_order ? 1 : 0));
  return EHC_OK;
}

int ehc_get_lattice_temperature(ehc_ctx *h, double *Tl_dev_out) {
  if (!h || (!Tl_dev_out && h->c.n > 0)) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.built) return EHC_E_STATE;
  CK(launch_unpermute(c, c.Tl_d, Tl_dev_out, 0));
  return EHC_OK;
}

int ehc_export_neighbors(ehc_ctx *h, int64_t *rowptr, int32_t *col, int64_t cap) {
  if (!h || !rowptr || (!col && cap > 0)) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.built) return EHC_E_STATE;
  const int64_t n = c.n;
  const int32_t w = c.n_max < c.W ? c.n_max : c.W;
  std::vector<uint8_t> cnt(n);
  std::vector<int32_t> perm(n), nbr((size_t)w * n);
  if (n > 0) {
    CK(cudaMemcpyAsync(cnt.data(), c.cnt, n, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(perm.data(), c.perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c.stream));
    if (w > 0)
      CK(cudaMemcpyAsync(nbr.data(), c.nbr, sizeof(int32_t) * (size_t)w * n, cudaMemcpyDeviceToHost, c.stream));
  }
  CK(cudaStreamSynchronize(c.stream));
  std::vector<int32_t> inv(n);
  for (int64_t s = 0; s < n; ++s) inv[perm[s]] = (int32_t)s;
  rowptr[0] = 0;
  for (int64_t o = 0; o < n; ++o) rowptr[o + 1] = rowptr[o] + cnt[inv[o]];
  if (rowptr[n] > cap) return EHC_E_INVAL;
  for (int64_t o = 0; o < n; ++o) {
    const int64_t s = inv[o];
    int64_t b = rowptr[o];
    for (int k = 0; k < cnt[s]; ++k) col[b + k] = perm[nbr[(size_t)k * n + s]];
    std::sort(col + b, col + b + cnt[s]);
  }
  return EHC_OK;
}

int ehc_md_step_host(ehc_ctx *h, double *x_host, double *v_host, int32_t n_sub, double t_fs, double dt_md_fs,
                     double *Te_host_out) {
  NvtxRange nvtx_range("ehc_md_step_host");
  if (!h || (h->c.n > 0 && (!x_host || !v_host || !Te_host_out))) return EHC_E_INVAL;
  Ctx &c = h->c;
  const size_t b3 = sizeof(double) * 3 * (size_t)c.n;
  if (!c.have_te) return EHC_E_STATE;
  if (c.n == 0) {
    int r = ehc_build_neighbors(h, c.x_dev, c.v_dev);
    if (r == EHC_OK) r = ehc_substep(h, n_sub, t_fs);
    if (r == EHC_OK) r = ehc_couple(h, c.v_dev, dt_md_fs);
    if (r == EHC_OK) r = ehc_drift(h, c.x_dev, c.v_dev, dt_md_fs);
    return r ? r : ehc_sync(h);
  }
  // the positions go first on the context stream; the velocities, needed only by
  // the velocity gather after the neighbour search, come on io_stream meanwhile
  CK(cudaEventRecord(c.io_ev[0], c.stream));
  CK(cudaStreamWaitEvent(c.io_stream, c.io_ev[0], 0));
  CK(cudaMemcpyAsync(c.x_dev, x_host, b3, cudaMemcpyHostToDevice, c.stream));
  CK(cudaMemcpyAsync(c.v_dev, v_host, b3, cudaMemcpyHostToDevice, c.io_stream));
  CK(cudaEventRecord(c.io_ev[1], c.io_stream));
  int r = build_enqueue(c, c.x_dev, c.v_dev, c.io_ev[1]);
  if (r) {
    cudaStreamSynchronize(c.io_stream);
    cudaStreamSynchronize(c.stream);
    return r;
  }
  CK(cudaStreamSynchronize(c.stream));
  r = build_finish(c, true);
  if (r) return r;
  r = ehc_substep(h, n_sub, t_fs);
  if (r) return r;
  r = ehc_couple(h, c.v_dev, dt_md_fs);
  if (r) return r;
  // the velocities are final after the hand-over: download them on io_stream
  // while the context stream runs the drift (which only reads them)
  CK(cudaEventRecord(c.io_ev[2], c.stream));
  CK(cudaStreamWaitEvent(c.io_stream, c.io_ev[2], 0));
  CK(cudaMemcpyAsync(v_host, c.v_dev, b3, cudaMemcpyDeviceToHost, c.io_stream));
  // T_e in caller order first, downloaded on io_stream while the context stream
  // runs the drift and downloads the positions
  r = ehc_get_te(h, c.T_out);
  if (r == EHC_OK) {
    CK(cudaEventRecord(c.io_ev[3], c.stream));
    CK(cudaStreamWaitEvent(c.io_stream, c.io_ev[3], 0));
    CK(cudaMemcpyAsync(Te_host_out, c.T_out, sizeof(double) * c.n, cudaMemcpyDeviceToHost, c.io_stream));
    r = ehc_drift(h, c.x_dev, c.v_dev, dt_md_fs);
  }
  if (r) {
    cudaStreamSynchronize(c.io_stream);
    return r;
  }
  CK(cudaMemcpyAsync(x_host, c.x_dev, b3, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.io_stream));
  return ehc_sync(h);
}

int ehc_philox_normals(const int64_t *ids_dev, int64_t n, uint64_t md_step, uint64_t seed, double *out_dev,
                       void *stream) {
  if (n < 0 || (n > 0 && (!ids_dev || !out_dev))) return EHC_E_INVAL;
  CK(launch_philox_normals(ids_dev, n, md_step, seed, out_dev, (cudaStream_t)stream));
  return EHC_OK;
}

// checkpoint file: magic, version, n, md_step, ledger scalars, T and A in caller order
namespace {
struct CkptHeader {
  char magic[8];
  int64_t version, n, md_step;
  double E_e0, E_base, ST_base, VC_prev, E_src, E_lat;
  uint64_t n_stopped, seed;
  int64_t flux_prec;
};
}  // namespace

int ehc_save(ehc_ctx *h, const char *path) {
  NvtxRange nvtx_range("ehc_save");
  if (!h || !path) return EHC_E_INVAL;
  Ctx &c = h->c;
  if (!c.have_te || c.has_border || c.border_next) return EHC_E_STATE;
  std::vector<double> T(c.n), A(c.n);
  int r = ehc_get_te(h, c.T_out);
  if (r) return r;
  if (c.n > 0) {
    CK(cudaMemcpyAsync(T.data(), c.T_out, sizeof(double) * c.n, cudaMemcpyDeviceToHost, c.stream));
    CK(launch_unpermute(c, c.A, c.T_out, c.te_orig_order ? 1 : 0));
    CK(cudaMemcpyAsync(A.data(), c.T_out, sizeof(double) * c.n, cudaMemcpyDeviceToHost, c.stream));
  }
  r = readback(c);
  if (r) return r;
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "EHCCKPT1", 8);
  hd.version = 1;
  hd.n = c.n;
  hd.md_step = c.md_step;
  hd.E_e0 = c.E_e0;
  hd.E_base = c.E_base;
  hd.ST_base = c.ST_base;
  hd.VC_prev = c.VC_prev;
  hd.E_src = c.E_src;
  hd.E_lat = c.scal_host[8];
  std::memcpy(&hd.n_stopped, c.scal_host + 9, sizeof(uint64_t));
  hd.seed = c.p.seed;
  hd.flux_prec = c.p.flux_prec;
  FILE *f = std::fopen(path, "wb");
  if (!f) return EHC_E_INVAL;
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
  if (c.n > 0) {
    ok = ok && std::fwrite(T.data(), sizeof(double), c.n, f) == (size_t)c.n;
    ok = ok && std::fwrite(A.data(), sizeof(double), c.n, f) == (size_t)c.n;
  }
  ok = (std::fclose(f) == 0) && ok;
  return ok ? EHC_OK : EHC_E_INVAL;
}

int ehc_load(ehc_ctx *h, const char *path) {
  NvtxRange nvtx_range("ehc_load");
  if (!h || !path) return EHC_E_INVAL;
  Ctx &c = h->c;
  c.t_version += 1;
  FILE *f = std::fopen(path, "rb");
  if (!f) return EHC_E_INVAL;
  CkptHeader hd;
  bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, "EHCCKPT1", 8) == 0 && hd.n == c.n &&
            hd.version == 1;
  std::vector<double> T(c.n), A(c.n);
  if (ok && c.n > 0) {
    ok = std::fread(T.data(), sizeof(double), c.n, f) == (size_t)c.n;
    ok = ok && std::fread(A.data(), sizeof(double), c.n, f) == (size_t)c.n;
  }
  std::fclose(f);
  if (!ok) return EHC_E_INVAL;
  if (c.n > 0) {
    CK(cudaMemcpyAsync(c.T[c.tcur], T.data(), sizeof(double) * c.n, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(c.A, A.data(), sizeof(double) * c.n, cudaMemcpyHostToDevice, c.stream));
  }
  c.scal_host[8] = hd.E_lat;
  std::memcpy(c.scal_host + 9, &hd.n_stopped, sizeof(uint64_t));
  CK(cudaMemcpyAsync(c.scal + 8, c.scal_host + 8, sizeof(double) * 2, cudaMemcpyHostToDevice, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  c.md_step = hd.md_step;
  c.E_e0 = hd.E_e0;
  c.E_base = hd.E_base;
  c.ST_base = hd.ST_base;
  c.VC_prev = hd.VC_prev;
  c.E_src = hd.E_src;
  c.p.seed = hd.seed;
  c.have_te = true;
  c.te_orig_order = true;
  c.built = false;
  c.ff_valid = false;
  c.t_stale = false;
  return EHC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched replicas: independent systems advanced together.  Every replica keeps
// its own context (neighbour list, coefficients, ledger); the substeps of all
// replicas run as one launch of the row-tile kernel per substep over a work list
// of (replica, row) items, replayed from a CUDA graph.

struct ehc_batch {
  std::vector<ehc_ctx *> rep;
  std::vector<int64_t> off;      // first atom of each replica in the concatenated arrays
  int64_t n_total = 0;
  ehc_params p;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  // per-replica work (builds, hand-over, drift) runs on kRepStreams streams,
  // replica r on rs[r % kRepStreams], forked from and joined back to `stream`
  std::vector<cudaStream_t> rs;
  std::vector<cudaEvent_t> rev;
  cudaEvent_t fork_ev = nullptr;
  RepArgs *reps_dev = nullptr;
  int2 *work = nullptr;
  int32_t nwork = 0, tile_floats = 0, num_sms = 0;
  int32_t tile_grid[2] = {0, 0}, tile_grid128[2] = {0, 0};
  int32_t tile_nt = 0;           // threads owning atoms chosen by the tuner (0: not tuned yet)
  int32_t tile_q = 4;            // persistent grid in quarters of the resident CTAs
  int parity = 0;
  struct G {
    int n_sub, parity, pairs, tile, nt;
    cudaGraphExec_t exec;
  };
  std::vector<G> graphs;
};

namespace {

constexpr int kRepStreams = 16;

// the replica streams wait for everything queued on the batch stream so far
cudaError_t batch_fork(ehc_batch &b) {
  cudaError_t e = cudaEventRecord(b.fork_ev, b.stream);
  for (size_t k = 0; k < b.rs.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b.rs[k], b.fork_ev, 0);
  return e;
}

// the batch stream waits for everything queued on the replica streams
cudaError_t batch_join(ehc_batch &b) {
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < b.rs.size() && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b.rev[k], b.rs[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b.stream, b.rev[k], 0);
  }
  return e;
}

int batch_pairs(const ehc_batch &b) {
  int pairs = 9;
  for (auto *h : b.rep) {
    const int P = (h->c.n_max + 1) / 2;
    if (P != 9) pairs = 16;
  }
  return pairs;
}

bool batch_tile_ok(const ehc_batch &b) {
  if (b.tile_floats <= 0 || b.nwork <= 0 || b.tile_grid[batch_pairs(b) == 9 ? 0 : 1] <= 0) return false;
  for (auto *h : b.rep)
    if (h->c.W > 32 || h->c.staged_max > b.tile_floats || h->c.p.flux_prec != 0) return false;
  return true;
}

}  // namespace

extern "C" {

int ehc_batch_create(const ehc_params *p, int32_t n_rep, const int64_t *n_atoms_host, const double *boxes_host,
                     const int32_t periodic[3], const double *mass_amu_host, void *stream, ehc_batch **out) {
  if (!p || n_rep <= 0 || !n_atoms_host || !boxes_host || !periodic || !mass_amu_host || !out) return EHC_E_INVAL;
  *out = nullptr;
  // batches use the row tiles: single precision, no source, uniform pair rates
  if (p->laser_on || p->flux_prec != 0 || p->rate_shell_n != 0 || p->ce_mode != 0) return EHC_E_INVAL;
  ehc_batch *b = new (std::nothrow) ehc_batch();
  if (!b) return EHC_E_NOMEM;
  b->p = *p;
  b->stream = (cudaStream_t)stream;
  const int ns = n_rep < kRepStreams ? n_rep : kRepStreams;
  bool sok = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < ns && sok; ++k) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    sok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    if (sok) b->rs.push_back(st);
    sok = sok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (sok) b->rev.push_back(ev);
  }
  if (!sok) {
    cudaGetLastError();
    ehc_batch_destroy(b);
    return EHC_E_NOMEM;
  }
  std::vector<int2> wl;
  for (int32_t r = 0; r < n_rep; ++r) {
    ehc_ctx *h = nullptr;
    int e = ehc_create(p, n_atoms_host[r], boxes_host + 3 * r, periodic, mass_amu_host, 1, nullptr,
                       b->rs[r % ns], &h);
    if (e != EHC_OK) {
      ehc_batch_destroy(b);
      return e;
    }
    b->rep.push_back(h);
    b->off.push_back(b->n_total);
    b->n_total += n_atoms_host[r];
    for (int64_t R = 0; R < h->c.nrows; ++R) wl.push_back(make_int2(r, (int)R));
  }
  b->nwork = (int32_t)wl.size();
  bool ok = cudaMalloc((void **)&b->reps_dev, sizeof(RepArgs) * n_rep) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&b->work, sizeof(int2) * (wl.empty() ? 1 : wl.size())) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, 0) == cudaSuccess;
  if (ok && !wl.empty())
    ok = cudaMemcpy(b->work, wl.data(), sizeof(int2) * wl.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ehc_batch_destroy(b);
    return EHC_E_NOMEM;
  }
  *out = b;
  return EHC_OK;
}

void ehc_batch_destroy(ehc_batch *b) {
  if (!b) return;
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
  for (auto *h : b->rep) ehc_destroy(h);
  if (b->reps_dev) cudaFree(b->reps_dev);
  if (b->work) cudaFree(b->work);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (auto st : b->rs) cudaStreamDestroy(st);
  for (auto ev : b->rev) cudaEventDestroy(ev);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  delete b;
}

int ehc_batch_size(const ehc_batch *b, int64_t *n_total, int64_t *offsets_host) {
  if (!b) return EHC_E_INVAL;
  if (n_total) *n_total = b->n_total;
  if (offsets_host)
    for (size_t r = 0; r < b->off.size(); ++r) offsets_host[r] = b->off[r];
  return EHC_OK;
}

int ehc_batch_set_te(ehc_batch *b, const double *Te_dev) {
  if (!b || (!Te_dev && b->n_total > 0)) return EHC_E_INVAL;
  CK(batch_fork(*b));
  for (size_t r = 0; r < b->rep.size(); ++r) {
    int e = ehc_set_te(b->rep[r], Te_dev + b->off[r]);
    if (e) return e;
  }
  CK(batch_join(*b));
  b->parity = 0;
  return EHC_OK;
}

int ehc_batch_build_neighbors(ehc_batch *b, const double *x_dev, const double *v_dev) {
  NvtxRange nvtx_range("ehc_batch_build_neighbors");
  if (!b || (b->n_total > 0 && (!x_dev || !v_dev))) return EHC_E_INVAL;
  CK(batch_fork(*b));
  for (size_t r = 0; r < b->rep.size(); ++r) {
    int e = build_enqueue(b->rep[r]->c, x_dev + 3 * b->off[r], v_dev + 3 * b->off[r]);
    if (e) return e;
  }
  CK(batch_join(*b));
  CK(cudaStreamSynchronize(b->stream));
  int first_err = EHC_OK;
  int32_t staged = 0;
  std::vector<RepArgs> tab(b->rep.size());
  for (size_t r = 0; r < b->rep.size(); ++r) {
    Ctx &c = b->rep[r]->c;
    int e = build_finish(c, false);
    if (e && !first_err) first_err = e;
    staged = std::max(staged, c.staged_max);
    tab[r] = rep_args(c);
  }
  if (staged > b->tile_floats) {
    int32_t tb = 0, grid[2] = {0, 0}, grid128[2] = {0, 0};
    if (tile_size(staged, b->num_sms, &tb, grid, grid128)) {
      b->tile_floats = tb;
      b->tile_nt = 0;
      b->tile_grid128[0] = grid128[0];
      b->tile_grid128[1] = grid128[1];
      b->tile_grid[0] = grid[0];
      b->tile_grid[1] = grid[1];
    }
  }
  CK(cudaMemcpy(b->reps_dev, tab.data(), sizeof(RepArgs) * tab.size(), cudaMemcpyHostToDevice));
  CK(batch_join(*b));   // the coefficient uploads of build_finish
  b->parity = 0;
  return first_err;
}

int ehc_batch_substep(ehc_batch *b, int32_t n_sub, double t_fs) {
  NvtxRange nvtx_range("ehc_batch_substep");
  if (!b || n_sub < 0) return EHC_E_INVAL;
  for (auto *h : b->rep) {
    if (!h->c.built) return EHC_E_STATE;
    if (h->c.n > 0 && !(h->c.stability <= 2.0)) return EHC_E_UNSTABLE;
  }
  if (n_sub == 0) return EHC_OK;
  CK(batch_fork(*b));
  if (!batch_tile_ok(*b)) {
    // some replica does not fit the row tiles: advance each on its own
    for (auto *h : b->rep) {
      int e = ehc_substep(h, n_sub, t_fs);
      if (e) return e;
    }
    CK(batch_join(*b));
    return EHC_OK;
  }
  for (auto *h : b->rep) {
    h->c.parity = b->parity;
    int e = ensure_split(h->c);
    if (e) return e;
  }
  CK(batch_join(*b));
  const int p0 = b->parity;
  const int pairs = batch_pairs(*b);
  const int pw = pairs == 9 ? 0 : 1;
  int32_t rest = n_sub;
  if (b->p.tile_threads) {
    b->tile_nt = b->p.tile_threads;
    b->tile_q = b->p.tile_grid_quarters ? b->p.tile_grid_quarters : 4;
  }
  auto share = [](int32_t g, int32_t q) { return g * q / 4 > 0 ? g * q / 4 : 1; };
  if (b->tile_nt == 0 && n_sub >= 2 * kTuneCands + 4 && b->tile_grid128[pw] > 0) {
    int32_t chosen = 256, q = 4;
    int r = tune_tiles(b->stream, &chosen, &q, [&](int k, int nt, int qq) {
      return launch_tile_worklist(b->reps_dev, b->work, b->nwork, b->tile_floats,
                                  share(nt == 128 ? b->tile_grid128[pw] : b->tile_grid[pw], qq), pairs,
                                  p0 ^ (k & 1), k, nt, b->stream);
    });
    if (r) return r;
    b->tile_nt = chosen;
    b->tile_q = q;
    rest -= 2 * kTuneCands;   // an even count: the mirror parity is unchanged
  }
  const int nt = b->tile_nt == 128 ? 128 : 256;
  const int32_t tgrid = share(nt == 128 ? b->tile_grid128[pw] : b->tile_grid[pw], b->tile_q);
  const int ntkey = nt * 8 + b->tile_q;
  int hit = -1;
  for (size_t i = 0; i < b->graphs.size(); ++i) {
    const auto &g = b->graphs[i];
    if (g.n_sub == rest && g.parity == p0 && g.pairs == pairs && g.tile == b->tile_floats && g.nt == ntkey)
      hit = (int)i;
  }
  if (hit < 0) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < rest && le == cudaSuccess; ++k)
      le = launch_tile_worklist(b->reps_dev, b->work, b->nwork, b->tile_floats, tgrid, pairs, p0 ^ (k & 1), k, nt,
                                b->cap_stream);
    cudaError_t ee = cudaStreamEndCapture(b->cap_stream, &graph);
    if (le != cudaSuccess || ee != cudaSuccess) return EHC_E_CUDA;
    cudaGraphExec_t exec;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return EHC_E_CUDA;
    if (b->graphs.size() >= 8) {
      cudaGraphExecDestroy(b->graphs.front().exec);
      b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back({rest, p0, pairs, b->tile_floats, ntkey, exec});
    hit = (int)b->graphs.size() - 1;
  }
  CK(cudaGraphLaunch(b->graphs[hit].exec, b->stream));
  b->parity = p0 ^ (n_sub & 1);
  for (auto *h : b->rep) {
    h->c.parity = b->parity;
    h->c.t_stale = true;
  }
  return EHC_OK;
}

int ehc_batch_couple(ehc_batch *b, double *v_dev, double dt_md_fs) {
  NvtxRange nvtx_range("ehc_batch_couple");
  if (!b || (b->n_total > 0 && !v_dev)) return EHC_E_INVAL;
  CK(batch_fork(*b));
  for (size_t r = 0; r < b->rep.size(); ++r) {
    int e = ehc_couple(b->rep[r], v_dev + 3 * b->off[r], dt_md_fs);
    if (e) return e;
  }
  CK(batch_join(*b));
  return EHC_OK;
}

int ehc_batch_drift(ehc_batch *b, double *x_dev, const double *v_dev, double dt_fs) {
  NvtxRange nvtx_range("ehc_batch_drift");
  if (!b || (b->n_total > 0 && (!x_dev || !v_dev))) return EHC_E_INVAL;
  CK(batch_fork(*b));
  for (size_t r = 0; r < b->rep.size(); ++r) {
    int e = ehc_drift(b->rep[r], x_dev + 3 * b->off[r], v_dev + 3 * b->off[r], dt_fs);
    if (e) return e;
  }
  CK(batch_join(*b));
  return EHC_OK;
}

int ehc_batch_get_te(ehc_batch *b, double *Te_dev_out) {
  if (!b || (b->n_total > 0 && !Te_dev_out)) return EHC_E_INVAL;
  CK(batch_fork(*b));
  for (size_t r = 0; r < b->rep.size(); ++r) {
    int e = ehc_get_te(b->rep[r], Te_dev_out + b->off[r]);
    if (e) return e;
  }
  CK(batch_join(*b));
  return EHC_OK;
}

int ehc_batch_energy(ehc_batch *b, int32_t r, ehc_energy_t *out) {
  if (!b || r < 0 || r >= (int32_t)b->rep.size()) return EHC_E_INVAL;
  CK(batch_fork(*b));
  return ehc_energy(b->rep[r], out);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Chebyshev window propagator

struct ehc_gnn;
namespace ehc {
int gnn_correct_window(ehc_gnn *g, Ctx &c, double kappa, float *ys, double *T1);
}

struct ehc_cheb {
  ehc_gnn *corr = nullptr;   // learned corrector applied to every window's result (or none)
  int n_w = 16, s = 4, order = 1;
  double eps = 0.05;
  int64_t n = 0;
  std::vector<double> nu, mut, kap, gam;   // stage coefficients, index 1..s
  float *y[4] = {nullptr, nullptr, nullptr, nullptr};   // stage values (padded to ps floats)
  float *z[3] = {nullptr, nullptr, nullptr};   // the window's change Y_j - Y_0 of the last three stages
  float *F0 = nullptr, *F1 = nullptr, *part = nullptr, *rho = nullptr, *host = nullptr;
  float *rr[2] = {nullptr, nullptr};   // row value ranges of the stage values
  double *T1 = nullptr, *dTc = nullptr;
  int64_t windows = 0, fallbacks = 0;
  // the row ranges of the state the next window starts from are in rr[rr_par]
  // if the previous window was accepted and no build came in between
  int64_t rr_build = -1;
  int rr_par = 0;
  // y[y0_buf] holds the values of the context's state while t_version == y0_version
  int64_t y0_version = -1;
  int y0_buf = 0;
  // training of the coefficients (allocated at the first train or predict call):
  // Adam on the relative changes d of the coefficients from `base`, c = base (1 + d)
  std::vector<double> base[4];          // nu, mut, kap, gam at the last set (or creation)
  float *tbuf = nullptr;                // y0 | z[1..s] | F[1..s] | lam[1..s], n floats each
  double *tT0 = nullptr, *tT1 = nullptr, *tlpart = nullptr, *tdpart = nullptr;
  float *tp = nullptr, *tm = nullptr, *tv = nullptr, *tgc = nullptr, *tgd = nullptr;
  float *tc0 = nullptr, *tloss = nullptr;
  float *thost = nullptr;               // pinned: c0[np] | loss | gc[np] | d[np]
  int adam_t = 0;
  std::vector<double> dacc;             // the accepted relative changes
  // rollout training (ehc_cheb_train_rollout), for up to ro_cap windows
  float *ro_buf = nullptr;              // window starts | per window z[1..s], F[1..s] | 5 work vectors
  double *ro_T = nullptr, *ro_lpart = nullptr;
  int ro_cap = 0;
  double x_spec = 0.0;                  // largest tau_w K |lambda_max| estimated so far (0: none)
};

namespace {

// Chebyshev polynomial T_j and its first two derivatives at x (three-term
// recurrence T_j = 2x T_{j-1} - T_{j-2}, differentiated)
void cheb_eval(int j, double x, double *T, double *dT, double *ddT) {
  double t0 = 1.0, t1 = x, d0 = 0.0, d1 = 1.0, e0 = 0.0, e1 = 0.0;
  if (j == 0) {
    *T = 1.0;
    *dT = 0.0;
    *ddT = 0.0;
    return;
  }
  for (int k = 1; k < j; ++k) {
    const double t2 = 2.0 * x * t1 - t0, d2 = 2.0 * t1 + 2.0 * x * d1 - d0, e2 = 4.0 * d1 + 2.0 * x * e1 - e0;
    t0 = t1;
    t1 = t2;
    d0 = d1;
    d1 = d2;
    e0 = e1;
    e1 = e2;
  }
  *T = t1;
  *dT = d1;
  *ddT = e1;
}

// Damped Chebyshev stage coefficients, w0 = 1 + eps/s^2.
// order 1: w1 = T_s/T_s', b_j = 1/T_j; mut_1 = w1/w0, nu_j = -b_j/b_{j-2},
//          mut_j = 2 w1 b_j/b_{j-1}, kap = gam = 0.
// order 2: w1 = T_s'/T_s'', b_j = T_j''/T_j'^2 (b_0 = b_1 = b_2),
//          a_j = 1 - b_j T_j; mut_1 = b_1 w1, mu_j = 2 b_j w0/b_{j-1},
//          nu_j = -b_j/b_{j-2}, mut_j = 2 b_j w1/b_{j-1}, kap_j = 1 - mu_j - nu_j,
//          gam_j = -a_{j-1} mut_j.  (All at w0.)
void cheb_coefficients(int s, int order, double eps, ehc_cheb *w) {
  const double w0 = 1.0 + eps / ((double)s * s);
  std::vector<double> T(s + 1), d1(s + 1), d2(s + 1), b(s + 1);
  for (int j = 0; j <= s; ++j) cheb_eval(j, w0, &T[j], &d1[j], &d2[j]);
  w->nu.assign(s + 1, 0.0);
  w->mut.assign(s + 1, 0.0);
  w->kap.assign(s + 1, 0.0);
  w->gam.assign(s + 1, 0.0);
  if (order == 1) {
    const double w1 = T[s] / d1[s];
    for (int j = 0; j <= s; ++j) b[j] = 1.0 / T[j];
    w->mut[1] = w1 / w0;
    for (int j = 2; j <= s; ++j) {
      w->nu[j] = -b[j] / b[j - 2];
      w->mut[j] = 2.0 * w1 * b[j] / b[j - 1];
    }
    return;
  }
  const double w1 = d1[s] / d2[s];
  for (int j = 2; j <= s; ++j) b[j] = d2[j] / (d1[j] * d1[j]);
  b[0] = b[1] = b[2];
  w->mut[1] = b[1] * w1;
  for (int j = 2; j <= s; ++j) {
    const double mu = 2.0 * b[j] * w0 / b[j - 1];
    w->nu[j] = -b[j] / b[j - 2];
    w->mut[j] = 2.0 * b[j] * w1 / b[j - 1];
    w->kap[j] = 1.0 - mu - w->nu[j];
    w->gam[j] = -(1.0 - b[j - 1] * T[j - 1]) * w->mut[j];
  }
}

// ---- training helpers ----
int cheb_np(const ehc_cheb *w) { return 4 * (w->s + 1); }

const std::vector<double> &cheb_set(const ehc_cheb *w, int q) {
  return q == 0 ? w->nu : (q == 1 ? w->mut : (q == 2 ? w->kap : w->gam));
}

std::vector<double> &cheb_set(ehc_cheb *w, int q) {
  return q == 0 ? w->nu : (q == 1 ? w->mut : (q == 2 ? w->kap : w->gam));
}

// P(x) of the stages on the linear test mode tau K F(Y) = -x Y (Y_0 = 1)
double cheb_poly(const ehc_cheb *w, double x) {
  double z2 = 0.0, z1 = -w->mut[1] * x;
  for (int j = 2; j <= w->s; ++j) {
    const double z = z1 + w->nu[j] * (z2 - z1) - w->kap[j] * z1 - w->mut[j] * x * (1.0 + z1) - w->gam[j] * x;
    z2 = z1;
    z1 = z;
  }
  return 1.0 + z1;
}

// coefficients base (1 + d), then mut and gam scaled so that P'(0) = -1
// (c_j = -dz_j/dx at x = 0: c_1 = mut_1, c_j = (1 - nu_j - kap_j) c_{j-1} + nu_j c_{j-2}
// + mut_j + gam_j, linear in (mut, gam)); d is rewritten to match
void cheb_apply(ehc_cheb *w, std::vector<double> &d) {
  const int s = w->s, S1 = s + 1;
  for (int b = 0; b < cheb_np(w); ++b) cheb_set(w, b / S1)[b % S1] = w->base[b / S1][b % S1] * (1.0 + d[b]);
  double c2 = 0.0, c1 = w->mut[1];
  for (int j = 2; j <= s; ++j) {
    const double cj = (1.0 - w->nu[j] - w->kap[j]) * c1 + w->nu[j] * c2 + w->mut[j] + w->gam[j];
    c2 = c1;
    c1 = cj;
  }
  if (std::isfinite(c1) && c1 > 0.0)
    for (int j = 1; j <= s; ++j) {
      w->mut[j] /= c1;
      w->gam[j] /= c1;
    }
  for (int b = 0; b < cheb_np(w); ++b) {
    const double bs = w->base[b / S1][b % S1];
    d[b] = bs != 0.0 ? cheb_set(w, b / S1)[b % S1] / bs - 1.0 : 0.0;
  }
}

// stability check of training: |P| <= 1 + kStabTol on a grid of kStabGrid points
// (the sampling misses a peak between points by at most s^2 (2 dx / X)^2 / 2,
// about 2e-6 for 16 stages on X = 140)
constexpr int kStabGrid = 16384;
constexpr double kStabTol = 1e-6;

// max over x_k = xmax k / npts (k = 1..npts) of |P(x_k)| - 1
double cheb_violation(const ehc_cheb *w, double xmax, int npts) {
  double v = -1.0;
  for (int k = 1; k <= npts; ++k) {
    const double P = std::fabs(cheb_poly(w, xmax * k / npts)) - 1.0;
    v = std::isfinite(P) ? std::max(v, P) : 1e300;
  }
  return v;
}

int cheb_train_prepare(ehc_cheb *w, Ctx &c) {
  if (w->tbuf) return EHC_OK;
  const int s = w->s, np = cheb_np(w);
  const int64_t n = c.n > 0 ? c.n : 1;
  bool ok = true;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  A(dalloc(&w->tbuf, n * (1 + 3 * (int64_t)s)));
  A(dalloc(&w->tT0, n));
  A(dalloc(&w->tT1, n));
  A(dalloc(&w->tlpart, (int64_t)wt_loss_partials(n)));
  A(dalloc(&w->tdpart, (int64_t)wt_dot_partials(n, s)));
  for (float **q : {&w->tp, &w->tm, &w->tv, &w->tgc, &w->tgd, &w->tc0}) A(dalloc(q, np));
  A(dalloc(&w->tloss, 1));
  A(cudaMallocHost((void **)&w->thost, sizeof(float) * (3 * np + 1)));
  if (ok) {
    for (float *q : {w->tp, w->tm, w->tv}) A(cudaMemsetAsync(q, 0, sizeof(float) * np, c.stream));
    for (int b = 0; b < np; ++b) w->thost[b] = (float)w->base[b / (s + 1)][b % (s + 1)];
    A(cudaMemcpyAsync(w->tc0, w->thost, sizeof(float) * np, cudaMemcpyHostToDevice, c.stream));
    A(cudaStreamSynchronize(c.stream));
  }
  if (!ok) {
    cudaGetLastError();
    return EHC_E_NOMEM;
  }
  w->adam_t = 0;
  w->dacc.assign(np, 0.0);
  return EHC_OK;
}

WtTab cheb_train_tab(const ehc_cheb *w, int64_t n) {
  WtTab t{};
  for (int j = 1; j <= w->s; ++j) {
    t.z[j] = w->tbuf + n * j;
    t.F[j] = w->tbuf + n * (w->s + j);
    t.lam[j] = w->tbuf + n * (2 * w->s + j);
  }
  return t;
}

// after a backward pass (loss in w->tloss, gradients in w->tgc / w->tgd): the
// loss and gradient to the host and, if lr > 0, the Adam step, projected to
// P'(0) = -1 (slow modes decay at the plain rate) and taken back by halves until
// |P| <= 1 on (0, xr] again
int cheb_step_tail(ehc_cheb *w, Ctx &c, float lr, double xr, float *loss_host, float *grad_host);

WtCoef cheb_train_coef(const ehc_cheb *w, const Ctx &c) {
  WtCoef k{};
  const double tauK = (double)w->n_w * c.p.dt_sub_fs * c.K;
  for (int j = 1; j <= w->s; ++j) {
    k.nu[j] = (float)w->nu[j];
    k.kap[j] = (float)w->kap[j];
    k.a[j] = (float)(w->mut[j] * tauK);
    k.g[j] = (float)(w->gam[j] * tauK);
  }
  return k;
}

int cheb_step_tail(ehc_cheb *w, Ctx &c, float lr, double xr, float *loss_host, float *grad_host) {
  const int np = cheb_np(w);
  float *hl = w->thost + np, *hg = w->thost + np + 1, *hd = w->thost + 2 * np + 1;
  CK(cudaMemcpyAsync(hl, w->tloss, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(hg, w->tgc, sizeof(float) * np, cudaMemcpyDeviceToHost, c.stream));
  if (lr > 0.0f) {
    w->adam_t += 1;
    CK(wt_adam(c.stream, np, w->tp, w->tm, w->tv, w->tgd, lr, w->adam_t));
    CK(cudaMemcpyAsync(hd, w->tp, sizeof(float) * np, cudaMemcpyDeviceToHost, c.stream));
  }
  CK(cudaStreamSynchronize(c.stream));
  if (loss_host) *loss_host = *hl;
  if (grad_host) std::memcpy(grad_host, hg, sizeof(float) * np);
  if (lr > 0.0f) {
    const std::vector<double> dold = w->dacc;
    std::vector<double> dtry(np);
    bool taken = false;
    double t = 1.0;
    for (int k = 0; k <= 20 && !taken; ++k, t *= 0.5) {
      for (int b = 0; b < np; ++b) dtry[b] = dold[b] + t * ((double)hd[b] - dold[b]);
      cheb_apply(w, dtry);
      taken = cheb_violation(w, xr, kStabGrid) <= kStabTol;
    }
    if (taken) {
      w->dacc = dtry;
    } else {
      dtry = dold;
      cheb_apply(w, dtry);
    }
    for (int b = 0; b < np; ++b) hd[b] = (float)w->dacc[b];
    CK(cudaMemcpyAsync(w->tp, hd, sizeof(float) * np, cudaMemcpyHostToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
  }
  return EHC_OK;
}

}  // namespace

extern "C" {

int ehc_cheb_create(ehc_ctx *hc, int32_t n_window, int32_t stages, int32_t order, double damping,
                    ehc_cheb **out) {
  if (!hc || !out || n_window < 1 || stages < 2 || stages > 32 || (order != 1 && order != 2) ||
      !(damping >= 0.0) || damping > 10.0)
    return EHC_E_INVAL;
  *out = nullptr;
  Ctx &c = hc->c;
  if (c.p.flux_prec != 0 || c.p.laser_on) return EHC_E_INVAL;
  ehc_cheb *w = new (std::nothrow) ehc_cheb();
  if (!w) return EHC_E_NOMEM;
  w->n_w = n_window;
  w->s = stages;
  w->order = order;
  w->eps = damping;
  w->n = c.n;
  cheb_coefficients(stages, order, damping, w);
  for (int q = 0; q < 4; ++q) w->base[q] = cheb_set(w, q);
  const int64_t n = c.n > 0 ? c.n : 1;
  const int64_t np4 = c.ps > 0 ? c.ps : 4;
  bool ok = true;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  for (int k = 0; k < 4; ++k) A(dalloc(&w->y[k], np4));
  for (int k = 0; k < 3; ++k) A(dalloc(&w->z[k], n));
  A(dalloc(&w->F0, n));
  A(dalloc(&w->F1, n));
  A(dalloc(&w->part, cheb_blocks(n)));
  A(dalloc(&w->rho, 1));
  A(dalloc(&w->T1, n));
  A(dalloc(&w->dTc, n));
  A(dalloc(&w->rr[0], 2 * (c.nrows > 0 ? c.nrows : 1)));
  A(dalloc(&w->rr[1], 2 * (c.nrows > 0 ? c.nrows : 1)));
  A(cudaMallocHost((void **)&w->host, sizeof(float) * 4));
  if (ok)
    for (int k = 0; k < 4; ++k) A(cudaMemsetAsync(w->y[k], 0, sizeof(float) * np4, c.stream));
  if (ok) A(cudaStreamSynchronize(c.stream));
  if (!ok) {
    cudaGetLastError();
    ehc_cheb_destroy(w);
    return EHC_E_NOMEM;
  }
  *out = w;
  return EHC_OK;
}

void ehc_cheb_destroy(ehc_cheb *w) {
  if (!w) return;
  for (int k = 0; k < 4; ++k)
    if (w->y[k]) cudaFree(w->y[k]);
  for (int k = 0; k < 3; ++k)
    if (w->z[k]) cudaFree(w->z[k]);
  void *p[] = {w->F0,  w->F1,     w->part,   w->rho, w->T1, w->dTc, w->rr[0], w->rr[1], w->tbuf,
               w->tT0, w->tT1,    w->tlpart, w->tdpart, w->tp, w->tm,  w->tv,    w->tgc,   w->tgd,
               w->tc0, w->tloss};
  for (void *q : p)
    if (q) cudaFree(q);
  if (w->host) cudaFreeHost(w->host);
  if (w->thost) cudaFreeHost(w->thost);
  for (void *q : {(void *)w->ro_buf, (void *)w->ro_T, (void *)w->ro_lpart})
    if (q) cudaFree(q);
  delete w;
}

int ehc_cheb_coefficients(const ehc_cheb *w, double *nu_out, double *mut_out, double *kap_out, double *gam_out) {
  if (!w || !nu_out || !mut_out) return EHC_E_INVAL;
  for (int j = 0; j <= w->s; ++j) {
    nu_out[j] = w->nu[j];
    mut_out[j] = w->mut[j];
    if (kap_out) kap_out[j] = w->kap[j];
    if (gam_out) gam_out[j] = w->gam[j];
  }
  return EHC_OK;
}

int ehc_cheb_step(ehc_cheb *w, ehc_ctx *hc, double tau, double t_fs, int32_t *fell_back, double *rho_out) {
  NvtxRange nvtx_range("ehc_cheb_step");
  if (!w || !hc || hc->c.n != w->n) return EHC_E_INVAL;
  Ctx &c = hc->c;
  if (!c.built) return EHC_E_STATE;
  if (!(c.stability <= 2.0)) return EHC_E_UNSTABLE;
  if (c.n == 0) return EHC_OK;
  if (!tile_path(c) || c.has_border) {
    // the stages run in the row-tile kernel and know no border; without it, or
    // with a border, advance the window plainly
    w->windows += 1;
    w->fallbacks += 1;
    if (fell_back) *fell_back = 1;
    if (rho_out) *rho_out = -1.0;
    return ehc_substep(hc, w->n_w, t_fs);
  }
  int r = ensure_t(c);
  if (r) return r;
  const double *T0 = c.T[c.tcur];
  double *T1 = c.T[c.tcur ^ 1];   // free outside builds and FP64 substeps; becomes the state on accept
  const double tauw = (double)w->n_w * c.p.dt_sub_fs;
  // Y_0 stays in y[b0] through the window (the second-order stages use it);
  // the stages rotate through the other three buffers.  Y_0 is the previous
  // window's end values if nothing touched T since, else made from T.
  int b0 = 0;
  if (w->y0_version == c.t_version) {
    b0 = w->y0_buf;
  } else {
    CK(cheb_mirror(c, T0, w->y[0]));
  }
  float *rot[3] = {w->y[(b0 + 1) & 3], w->y[(b0 + 2) & 3], w->y[(b0 + 3) & 3]};
  // row ranges of the first stage: those of the previous window's end state when
  // it was accepted since the last build, else unknown (widest tier)
  int par = 0;
  if (w->rr_build == c.builds && w->y0_version == c.t_version) {
    par = w->rr_par;
  } else {
    CK(cudaMemsetAsync(w->rr[0], 0xfe, sizeof(float) * c.nrows, c.stream));
    CK(cudaMemsetAsync(w->rr[0] + c.nrows, 0x7f, sizeof(float) * c.nrows, c.stream));
  }
  w->rr_build = -1;
  w->y0_version = -1;
  const float *Y0 = w->y[b0];
  // the F(Y_0) term of the later stages (second order, or trained coefficients)
  bool use_f0 = false;
  for (int j = 2; j <= w->s; ++j) use_f0 = use_f0 || w->gam[j] != 0.0;
  // the window's coupling factor 1 - (1 - dt G/C_e)^n_w, applied by the last stage
  const double fin = 1.0 - std::pow(1.0 - c.p.dt_sub_fs * c.cG, (double)w->n_w);
  for (int j = 1; j <= w->s; ++j) {
    StageArgs sa{};
    sa.yin = j == 1 ? Y0 : rot[(j - 2) % 3];
    sa.y0 = Y0;
    sa.zin = j >= 2 ? w->z[(j - 2) % 3] : nullptr;
    sa.zprev = j >= 3 ? w->z[(j - 3) % 3] : nullptr;
    sa.zout = w->z[(j - 1) % 3];
    sa.yout = rot[(j - 1) % 3];
    sa.Fout = j == 1 ? w->F0 : nullptr;
    sa.F0 = (use_f0 && j >= 2) ? w->F0 : nullptr;
    sa.rr[0] = w->rr[0];
    sa.rr[1] = w->rr[1];
    sa.nu = (float)w->nu[j];
    sa.mt = (float)(w->mut[j] * tauw * c.K);
    sa.kap = (float)w->kap[j];
    sa.gt = (float)(w->gam[j] * tauw * c.K);
    if (j == w->s) {
      // back to FP64 with the electron-phonon coupling of the window (kept in dTc until accepted)
      sa.T0 = T0;
      sa.T1 = T1;
      sa.dTc = w->dTc;
      sa.fin = (float)fin;
      sa.Tref_f = (float)c.p.Tref_K;
      sa.invTmax_f = (float)(1.0 / c.p.Tmax_K);
      sa.Tmax = c.p.Tmax_K;
    }
    CK(launch_cheb_stage(c, sa, par, c.stream));
    par ^= 1;
  }
  float *ys = rot[(w->s - 1) % 3];
  int bs = 0;
  for (int k = 0; k < 4; ++k)
    if (w->y[k] == ys) bs = k;
  // the learned corrector's pair flux on the window's result (T1 and its mirror)
  if (w->corr) {
    const int rc = gnn_correct_window(w->corr, c, tauw * c.K, ys, T1);
    if (rc) return rc;
  }
  // pair flux of the end state for the residual
  StageArgs sf{};
  sf.yin = ys;
  sf.y0 = ys;
  sf.zin = nullptr;
  sf.zprev = nullptr;
  sf.F0 = nullptr;
  sf.yout = nullptr;   // only the flux (and the row ranges of ys) is kept
  sf.zout = nullptr;
  sf.Fout = w->F1;
  sf.kap = 0.0f;
  sf.gt = 0.0f;
  sf.rr[0] = w->rr[0];
  sf.rr[1] = w->rr[1];
  sf.nu = 0.0f;
  sf.mt = 0.0f;
  CK(launch_cheb_stage(c, sf, par, c.stream));
  CK(cheb_residual(c, T0, T1, w->F0, w->F1, tauw, w->part, w->rho));
  CK(cudaMemcpyAsync(w->host, w->rho, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  const double rho = w->host[0];
  w->windows += 1;
  if (rho_out) *rho_out = rho;
  if (rho <= tau) {
    CK(cheb_accept(c, w->dTc));
    c.tcur ^= 1;
    c.ff_valid = false;
    c.t_stale = false;
    c.t_version += 1;
    // ys is the state's mirror; the flux pass recorded its row ranges
    w->y0_version = c.t_version;
    w->y0_buf = bs;
    w->rr_build = c.builds;
    w->rr_par = par ^ 1;
    if (fell_back) *fell_back = 0;
    return EHC_OK;
  }
  w->fallbacks += 1;
  if (fell_back) *fell_back = 1;
  return ehc_substep(hc, w->n_w, t_fs);
}

int ehc_cheb_stats(const ehc_cheb *w, int64_t *windows, int64_t *fallbacks) {
  if (!w) return EHC_E_INVAL;
  if (windows) *windows = w->windows;
  if (fallbacks) *fallbacks = w->fallbacks;
  return EHC_OK;
}

int ehc_cheb_set_coefficients(ehc_cheb *w, ehc_ctx *hc, const double *nu_host, const double *mut_host,
                              const double *kap_host, const double *gam_host) {
  if (!w || !hc || hc->c.n != w->n || !nu_host || !mut_host || !kap_host || !gam_host) return EHC_E_INVAL;
  const double *src[4] = {nu_host, mut_host, kap_host, gam_host};
  for (int q = 0; q < 4; ++q)
    for (int j = 0; j <= w->s; ++j)
      if (!std::isfinite(src[q][j]) || std::fabs(src[q][j]) > 1e6) return EHC_E_INVAL;
  Ctx &c = hc->c;
  for (int q = 0; q < 4; ++q) {
    cheb_set(w, q).assign(src[q], src[q] + w->s + 1);
    cheb_set(w, q)[0] = 0.0;
    w->base[q] = cheb_set(w, q);
  }
  // stage 1 is Y_1 = Y_0 + mut_1 tau K F(Y_0): its nu, kap and gam are unused
  for (int q : {0, 2, 3}) w->base[q][1] = cheb_set(w, q)[1] = 0.0;
  if (w->tbuf) {
    const int np = cheb_np(w);
    for (float *q : {w->tp, w->tm, w->tv}) CK(cudaMemsetAsync(q, 0, sizeof(float) * np, c.stream));
    for (int b = 0; b < np; ++b) w->thost[b] = (float)w->base[b / (w->s + 1)][b % (w->s + 1)];
    CK(cudaMemcpyAsync(w->tc0, w->thost, sizeof(float) * np, cudaMemcpyHostToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    w->adam_t = 0;
    w->dacc.assign(np, 0.0);
  }
  return EHC_OK;
}

int ehc_cheb_train_step(ehc_cheb *w, ehc_ctx *hc, const double *Tin_dev, const double *Ttar_dev, float lr,
                        int32_t loss_power, float *loss_host, float *grad_host) {
  NvtxRange nvtx_range("ehc_cheb_train_step");
  if (!w || !hc || hc->c.n != w->n || (hc->c.n > 0 && (!Tin_dev || !Ttar_dev)) || !(lr >= 0.0f) ||
      (loss_power != 2 && loss_power != 4 && loss_power != 8) || hc->c.p.rate_shell_n != 0 || hc->c.local)
    return EHC_E_INVAL;
  Ctx &c = hc->c;
  if (!c.built) return EHC_E_STATE;
  const int s = w->s, np = cheb_np(w);
  if (c.n == 0) {
    if (loss_host) *loss_host = 0.0f;
    if (grad_host) std::memset(grad_host, 0, sizeof(float) * np);
    return EHC_OK;
  }
  int r = cheb_train_prepare(w, c);
  if (r) return r;
  // stability range: 1.1 x the estimate of tau_w K |lambda_max| if one was made
  // (ehc_cheb_spectrum), else 1.1 x the bound n_w x the per-substep stability number
  const double xr = 1.1 * (w->x_spec > 0.0 ? w->x_spec : (double)w->n_w * c.stability);
  if (lr > 0.0f && cheb_violation(w, xr, kStabGrid) > kStabTol) return EHC_E_UNSTABLE;
  const WtTab t = cheb_train_tab(w, c.n);
  const WtCoef k = cheb_train_coef(w, c);
  const double tauK = (double)w->n_w * c.p.dt_sub_fs * c.K;
  float *y0 = w->tbuf;
  CK(nn_gather(c, Tin_dev, Ttar_dev, w->tT0, w->tT1, y0, false));
  CK(wt_stages(c, s, k, y0, t));
  CK(wt_backward(c, s, k, y0, t, w->tT0, w->tT1, loss_power, w->tlpart, w->tdpart, tauK, w->tc0, w->tgc, w->tgd,
                 w->tloss));
  return cheb_step_tail(w, c, lr, xr, loss_host, grad_host);
}

int ehc_cheb_train_rollout(ehc_cheb *w, ehc_ctx *hc, const double *Tin_dev, const double *Ttar_dev, int32_t n_win,
                           float lr, int32_t loss_power, float *loss_host, float *grad_host) {
  NvtxRange nvtx_range("ehc_cheb_train_rollout");
  if (!w || !hc || hc->c.n != w->n || (hc->c.n > 0 && (!Tin_dev || !Ttar_dev)) || n_win < 1 || n_win > 64 ||
      !(lr >= 0.0f) || (loss_power != 2 && loss_power != 4 && loss_power != 8) || hc->c.p.rate_shell_n != 0 || hc->c.local)
    return EHC_E_INVAL;
  Ctx &c = hc->c;
  if (!c.built) return EHC_E_STATE;
  const int s = w->s, np = cheb_np(w);
  if (c.n == 0) {
    if (loss_host) *loss_host = 0.0f;
    if (grad_host) std::memset(grad_host, 0, sizeof(float) * np);
    return EHC_OK;
  }
  int r = cheb_train_prepare(w, c);
  if (r) return r;
  const double xr = 1.1 * (w->x_spec > 0.0 ? w->x_spec : (double)w->n_w * c.stability);
  if (lr > 0.0f && cheb_violation(w, xr, kStabGrid) > kStabTol) return EHC_E_UNSTABLE;
  const int64_t n = c.n;
  if (n_win > w->ro_cap) {
    for (void *q : {(void *)w->ro_buf, (void *)w->ro_T, (void *)w->ro_lpart})
      if (q) cudaFree(q);
    w->ro_buf = nullptr;
    w->ro_T = w->ro_lpart = nullptr;
    w->ro_cap = 0;
    bool ok = true;
    auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
    A(dalloc(&w->ro_buf, n * ((int64_t)n_win + 1 + (int64_t)n_win * 2 * s + 5)));
    A(dalloc(&w->ro_T, n * (int64_t)n_win));
    A(dalloc(&w->ro_lpart, (int64_t)wt_loss_partials(n) * n_win));
    if (ok) A(cudaMemsetAsync(w->ro_buf, 0, sizeof(float) * n * ((int64_t)n_win + 1 + (int64_t)n_win * 2 * s + 5),
                              c.stream));
    if (!ok) {
      cudaGetLastError();
      return EHC_E_NOMEM;
    }
    w->ro_cap = n_win;
  }
  // layout within ro_buf (capacity ro_cap windows)
  const int cap = w->ro_cap;
  float *starts = w->ro_buf;
  float *zf = starts + n * (cap + 1);
  float *Lam = zf + n * (int64_t)cap * 2 * s;
  float *mu = Lam + n, *gs = mu + n, *tmp = gs + n, *zero = tmp + n;
  const WtTab t1 = cheb_train_tab(w, n);
  float *lam[kMaxStages + 1] = {};
  for (int j = 1; j <= s; ++j) lam[j] = const_cast<float *>(t1.lam[j]);
  std::vector<WtTab> tabs(n_win);
  std::vector<const float *> ys(n_win + 1);
  std::vector<const double *> Tt(n_win);
  for (int v = 0; v <= n_win; ++v) ys[v] = starts + n * v;
  for (int v = 0; v < n_win; ++v) {
    tabs[v] = WtTab{};
    for (int j = 1; j <= s; ++j) {
      tabs[v].z[j] = zf + n * ((int64_t)v * 2 * s + j - 1);
      tabs[v].F[j] = zf + n * ((int64_t)v * 2 * s + s + j - 1);
      tabs[v].lam[j] = lam[j];
    }
    Tt[v] = w->ro_T + n * v;
  }
  const WtCoef k = cheb_train_coef(w, c);
  const double tauK = (double)w->n_w * c.p.dt_sub_fs * c.K;
  // the start state and the targets in sorted order; then the windows, each from
  // the previous one's end
  CK(nn_gather(c, Tin_dev, nullptr, w->tT0, nullptr, starts, false));
  for (int v = 0; v < n_win; ++v) CK(nn_gather(c, Ttar_dev + n * v, nullptr, w->ro_T + n * v, nullptr, tmp, false));
  for (int v = 0; v < n_win; ++v) {
    CK(wt_stages(c, s, k, ys[v], tabs[v]));
    CK(wt_next_start(c, ys[v], tabs[v].z[s], const_cast<float *>(ys[v + 1])));
  }
  CK(wt_rollout(c, s, k, n_win, ys.data(), tabs.data(), Tt.data(), lam, Lam, mu, gs, tmp, zero, loss_power,
                w->ro_lpart, w->tdpart, tauK, w->tc0, w->tgc, w->tgd, w->tloss));
  return cheb_step_tail(w, c, lr, xr, loss_host, grad_host);
}

int ehc_cheb_spectrum(ehc_cheb *w, ehc_ctx *hc, const double *Tin_dev, int32_t iters, double *x_out) {
  if (!w || !hc || hc->c.n != w->n || iters < 1 || iters > 100000 || hc->c.p.rate_shell_n != 0 || hc->c.local) return EHC_E_INVAL;
  Ctx &c = hc->c;
  if (!c.built) return EHC_E_STATE;
  if (c.n == 0) {
    if (x_out) *x_out = 0.0;
    return EHC_OK;
  }
  int r = cheb_train_prepare(w, c);
  if (r) return r;
  const WtTab t = cheb_train_tab(w, c.n);
  float *y = w->tbuf;
  if (Tin_dev) {
    CK(nn_gather(c, Tin_dev, nullptr, w->tT0, nullptr, y, false));
  } else {
    r = ensure_t(c);
    if (r) return r;
    CK(cheb_mirror(c, c.T[c.tcur], y));
  }
  float *zero = const_cast<float *>(t.z[1]);
  CK(cudaMemsetAsync(zero, 0, sizeof(float) * c.n, c.stream));
  CK(wt_power(c, y, zero, const_cast<float *>(t.F[1]), const_cast<float *>(t.lam[1]), w->tdpart, w->tlpart,
              iters));
  double ss = 0.0;
  CK(cudaMemcpyAsync(&ss, w->tlpart, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  const double x = (double)w->n_w * c.p.dt_sub_fs * c.K * std::sqrt(ss);
  if (!std::isfinite(x)) return EHC_E_RANGE;
  w->x_spec = std::max(w->x_spec, x);
  if (x_out) *x_out = x;
  return EHC_OK;
}

int ehc_cheb_predict(ehc_cheb *w, ehc_ctx *hc, const double *Tin_dev, double *Tout_dev) {
  if (!w || !hc || hc->c.n != w->n || (hc->c.n > 0 && (!Tin_dev || !Tout_dev)) || hc->c.p.rate_shell_n != 0 || hc->c.local)
    return EHC_E_INVAL;
  Ctx &c = hc->c;
  if (!c.built) return EHC_E_STATE;
  if (c.n == 0) return EHC_OK;
  int r = cheb_train_prepare(w, c);
  if (r) return r;
  const WtTab t = cheb_train_tab(w, c.n);
  CK(nn_gather(c, Tin_dev, nullptr, w->tT0, nullptr, w->tbuf, false));
  CK(wt_stages(c, w->s, cheb_train_coef(w, c), w->tbuf, t));
  CK(wt_end(c, w->tT0, t.z[w->s], w->tT1));
  CK(launch_unpermute(c, w->tT1, Tout_dev, 0));
  return EHC_OK;
}

int ehc_cheb_stability(const ehc_cheb *w, double *beta) {
  if (!w || !beta) return EHC_E_INVAL;
  // no polynomial of degree s with P(0) = 1, P'(0) = -1 stays within [-1, 1]
  // beyond 2 s^2; scan a little past it
  constexpr int kScan = 200000;
  const double xlim = 2.05 * w->s * w->s, h = xlim / kScan;
  double good = 0.0;
  for (int k = 1; k <= kScan; ++k) {
    const double x = k * h;
    if (!(std::fabs(cheb_poly(w, x)) <= 1.0 + 1e-5)) break;
    good = x;
  }
  *beta = good;
  return EHC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned window propagator

struct ehc_nn {
  int H = 8, n_w = 16, np = 0;
  double sigma = 1e-3;
  int64_t n = 0;
  int t = 0;                       // Adam steps taken
  float *p = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
  __nv_bfloat16 *pb = nullptr, *h = nullptr;
  float *gphi = nullptr, *p1 = nullptr, *p2 = nullptr, *dm0 = nullptr, *dm1 = nullptr, *rpart = nullptr, *rho = nullptr;
  double *T0 = nullptr, *T1 = nullptr, *Ttar = nullptr;
  float *host = nullptr;           // pinned: loss, rho, gradient
  int64_t fallbacks = 0, windows = 0;
};

extern "C" {

int ehc_nn_create(ehc_ctx *hc, int32_t hidden, int32_t n_window, double sigma, ehc_nn **out) {
  if (!hc || !out || (hidden != 8 && hidden != 16) || n_window < 1 || !(sigma > 0)) return EHC_E_INVAL;
  *out = nullptr;
  Ctx &c = hc->c;
  if (c.p.flux_prec != 0 || c.p.laser_on || c.p.rate_shell_n != 0 || c.local) return EHC_E_INVAL;
  ehc_nn *nn = new (std::nothrow) ehc_nn();
  if (!nn) return EHC_E_NOMEM;
  nn->H = hidden;
  nn->n_w = n_window;
  nn->sigma = sigma;
  nn->n = c.n;
  nn->np = 8 * hidden + 1;
  const int64_t n = c.n > 0 ? c.n : 1;
  const int nb = nn_blocks(n);
  bool ok = true;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  A(dalloc(&nn->p, nn->np));
  A(dalloc(&nn->m, nn->np));
  A(dalloc(&nn->v, nn->np));
  A(dalloc(&nn->grad, nn->np));
  A(dalloc(&nn->loss, 1));
  A(dalloc(&nn->pb, nn->np));
  A(dalloc(&nn->h, n * hidden));
  A(dalloc(&nn->gphi, n));
  A(dalloc(&nn->p2, (int64_t)nb * (5 * hidden + 2)));
  A(dalloc(&nn->p1, (int64_t)nb * (3 * hidden)));
  A(dalloc(&nn->dm0, n));
  A(dalloc(&nn->dm1, n));
  A(dalloc(&nn->rpart, nb));
  A(dalloc(&nn->rho, 1));
  A(dalloc(&nn->T0, n));
  A(dalloc(&nn->T1, n));
  A(dalloc(&nn->Ttar, n));
  A(cudaMallocHost((void **)&nn->host, sizeof(float) * (nn->np + 4)));
  if (ok) {
    A(cudaMemsetAsync(nn->p, 0, sizeof(float) * nn->np, c.stream));
    A(cudaMemsetAsync(nn->m, 0, sizeof(float) * nn->np, c.stream));
    A(cudaMemsetAsync(nn->v, 0, sizeof(float) * nn->np, c.stream));
    A(cudaStreamSynchronize(c.stream));
  }
  if (!ok) {
    cudaGetLastError();
    ehc_nn_destroy(nn);
    return EHC_E_NOMEM;
  }
  *out = nn;
  return EHC_OK;
}

void ehc_nn_destroy(ehc_nn *nn) {
  if (!nn) return;
  void *d[] = {nn->p, nn->m, nn->v, nn->grad, nn->loss, nn->pb, nn->h, nn->gphi, nn->p1, nn->p2,
               nn->dm0, nn->dm1, nn->rpart, nn->rho, nn->T0, nn->T1, nn->Ttar};
  for (void *q : d)
    if (q) cudaFree(q);
  if (nn->host) cudaFreeHost(nn->host);
  delete nn;
}

int ehc_nn_set_params(ehc_nn *nn, ehc_ctx *hc, const float *params_host) {
  if (!nn || !hc || !params_host) return EHC_E_INVAL;
  Ctx &c = hc->c;
  CK(cudaMemcpyAsync(nn->p, params_host, sizeof(float) * nn->np, cudaMemcpyHostToDevice, c.stream));
  CK(cudaMemsetAsync(nn->m, 0, sizeof(float) * nn->np, c.stream));
  CK(cudaMemsetAsync(nn->v, 0, sizeof(float) * nn->np, c.stream));
  CK(nn_params_to_bf16(c.stream, nn->np, nn->p, nn->pb));
  CK(cudaStreamSynchronize(c.stream));
  nn->t = 0;
  return EHC_OK;
}

int ehc_nn_get_params(ehc_nn *nn, ehc_ctx *hc, float *params_host) {
  if (!nn || !hc || !params_host) return EHC_E_INVAL;
  Ctx &c = hc->c;
  CK(cudaMemcpyAsync(params_host, nn->p, sizeof(float) * nn->np, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  return EHC_OK;
}

int ehc_nn_train_step(ehc_nn *nn, ehc_ctx *hc, const double *Tin_dev, const double *Ttar_dev, float lr,
                      float *loss_host, float *grad_host) {
  NvtxRange nvtx_range("ehc_nn_train_step");
  if (!nn || !hc || (hc->c.n > 0 && (!Tin_dev || !Ttar_dev)) || hc->c.n != nn->n) return EHC_E_INVAL;
  Ctx &c = hc->c;
  if (!c.built) return EHC_E_STATE;
  CK(nn_gather(c, Tin_dev, Ttar_dev, nn->T0, nn->Ttar, nn->dm0, false));
  CK(nn_grad(c, nn->H, nn->pb, nn->sigma, nn->n_w, nn->dm0, nn->h, nn->T0, nn->Ttar, nn->gphi, nn->p2, nn->p1,
             nn->grad, nn->loss));
  CK(cudaMemcpyAsync(nn->host, nn->loss, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
  if (grad_host)
    CK(cudaMemcpyAsync(nn->host + 4, nn->grad, sizeof(float) * nn->np, cudaMemcpyDeviceToHost, c.stream));
  if (lr > 0.0f) {
    nn->t += 1;
    CK(nn_adam(c.stream, nn->np, nn->p, nn->m, nn->v, nn->grad, lr, nn->t, nn->pb));
  }
  CK(cudaStreamSynchronize(c.stream));
  if (loss_host) *loss_host = nn->host[0];
  if (grad_host) std::memcpy(grad_host, nn->host + 4, sizeof(float) * nn->np);
  return EHC_OK;
}

int ehc_nn_predict(ehc_nn *nn, ehc_ctx *hc, const double *Tin_dev, double *Tout_dev) {
  if (!nn || !hc || (hc->c.n > 0 && (!Tin_dev || !Tout_dev)) || hc->c.n != nn->n) return EHC_E_INVAL;
  Ctx &c = hc->c;
  if (!c.built) return EHC_E_STATE;
  CK(nn_gather(c, Tin_dev, nullptr, nn->T0, nullptr, nn->dm0, false));
  CK(nn_forward(c, nn->H, nn->pb, nn->sigma, nn->n_w, nn->dm0, nn->h, nn->T0, nn->T1, nn->dm1));
  CK(launch_unpermute(c, nn->T1, Tout_dev, 0));
  return EHC_OK;
}

int ehc_nn_step(ehc_nn *nn, ehc_ctx *hc, double tau, double t_fs, int32_t *fell_back, double *rho_out) {
  NvtxRange nvtx_range("ehc_nn_step");
  if (!nn || !hc || hc->c.n != nn->n) return EHC_E_INVAL;
  Ctx &c = hc->c;
  c.t_version += 1;
  if (!c.built) return EHC_E_STATE;
  if (!(c.stability <= 2.0)) return EHC_E_UNSTABLE;
  int r = ensure_t(c);
  if (r) return r;
  if (c.n == 0) return EHC_OK;
  if (c.has_border || c.local) {
    // the network knows neither a border nor the LOCAL form: plain substeps
    nn->windows += 1;
    nn->fallbacks += 1;
    if (fell_back) *fell_back = 1;
    if (rho_out) *rho_out = -1.0;
    return ehc_substep(hc, nn->n_w, t_fs);
  }
  // the window's state in sorted order: T0 and its mirror
  CK(nn_gather(c, c.T[c.tcur], nullptr, nn->T0, nullptr, nn->dm0, true));
  CK(nn_forward(c, nn->H, nn->pb, nn->sigma, nn->n_w, nn->dm0, nn->h, nn->T0, nn->T1, nn->dm1));
  CK(nn_couple_window(c, nn->T0, nn->T1, nn->dm1, nn->Ttar, nn->n_w));
  CK(nn_residual(c, nn->dm0, nn->dm1, nn->T0, nn->T1, (double)nn->n_w * c.p.dt_sub_fs, nn->rpart, nn->rho));
  CK(cudaMemcpyAsync(nn->host + 1, nn->rho, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  const double rho = nn->host[1];
  nn->windows += 1;
  if (rho_out) *rho_out = rho;
  if (rho <= tau) {
    CK(nn_accept(c, nn->Ttar));
    CK(cudaMemcpyAsync(c.T[c.tcur], nn->T1, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, c.stream));
    c.ff_valid = false;
    c.t_stale = false;
    if (fell_back) *fell_back = 0;
    return EHC_OK;
  }
  // residual above threshold: advance the window with the plain substeps
  nn->fallbacks += 1;
  if (fell_back) *fell_back = 1;
  return ehc_substep(hc, nn->n_w, t_fs);
}


}  // extern "C"

// ---- learned corrector of the window propagator (kernels_gnn.cu) ----

struct ehc_gnn {
  int64_t n = 0;
  double sigma = 1e-3;
  int t = 0;                      // Adam steps taken
  float *p = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  __nv_bfloat16 *pb = nullptr, *in = nullptr, *u = nullptr;
  float *y0 = nullptr, *ybuf = nullptr, *G = nullptr, *du = nullptr, *mpart = nullptr, *epart = nullptr;
  double *T = nullptr, *Tt = nullptr, *lpart = nullptr, *loss = nullptr;
  float *host = nullptr;          // pinned: gradient [kGnnParams] | loss
  double *host_loss = nullptr;
};

namespace ehc {
int gnn_correct_window(ehc_gnn *g, Ctx &c, double kappa, float *ys, double *T1) {
  if (g->n != c.n) return EHC_E_INVAL;
  CK(gnn_forward(c, g->pb, g->sigma, kappa, ys, g->in, g->u, T1, g->ybuf, nullptr));
  CK(cudaMemcpyAsync(ys, g->ybuf, sizeof(float) * c.n, cudaMemcpyDeviceToDevice, c.stream));
  return EHC_OK;
}
}  // namespace ehc

extern "C" {

int ehc_gnn_create(ehc_ctx *hc, double sigma, ehc_gnn **out) {
  if (!hc || !out || !(sigma > 0)) return EHC_E_INVAL;
  *out = nullptr;
  Ctx &c = hc->c;
  if (c.p.flux_prec != 0 || c.p.rate_shell_n != 0 || c.local) return EHC_E_INVAL;
  if (c.n > 2147483647LL) return EHC_E_INVAL;
  ehc_gnn *g = new (std::nothrow) ehc_gnn();
  if (!g) return EHC_E_NOMEM;
  g->n = c.n;
  g->sigma = sigma;
  const int64_t n = c.n > 0 ? c.n : 1;
  bool ok = gnn_setup(gnn_bwd_smem()) == cudaSuccess;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  A(dalloc(&g->p, kGnnParams));
  A(dalloc(&g->m, kGnnParams));
  A(dalloc(&g->v, kGnnParams));
  A(dalloc(&g->grad, kGnnParams));
  A(dalloc(&g->pb, kGnnParams));
  A(dalloc(&g->in, n * 16));
  A(dalloc(&g->u, n * 16));
  A(dalloc(&g->y0, n));
  A(dalloc(&g->ybuf, n));
  A(dalloc(&g->G, n));
  A(dalloc(&g->du, n * 16));
  A(dalloc(&g->mpart, (int64_t)gnn_mlp_blocks(c) * kGnnParams));
  A(dalloc(&g->epart, (int64_t)gnn_edge_blocks(n) * 64));
  A(dalloc(&g->T, n));
  A(dalloc(&g->Tt, n));
  A(dalloc(&g->lpart, gnn_loss_blocks(n)));
  A(dalloc(&g->loss, 1));
  A(cudaMallocHost((void **)&g->host, sizeof(float) * kGnnParams));
  A(cudaMallocHost((void **)&g->host_loss, sizeof(double)));
  if (ok) {
    // all parameters zero: the identity corrector until parameters are set
    A(cudaMemsetAsync(g->p, 0, sizeof(float) * kGnnParams, c.stream));
    A(cudaMemsetAsync(g->m, 0, sizeof(float) * kGnnParams, c.stream));
    A(cudaMemsetAsync(g->v, 0, sizeof(float) * kGnnParams, c.stream));
    A(gnn_params_to_bf16(c.stream, g->p, g->pb));
    A(cudaStreamSynchronize(c.stream));
  }
  if (!ok) {
    cudaGetLastError();
    ehc_gnn_destroy(g);
    return EHC_E_NOMEM;
  }
  *out = g;
  return EHC_OK;
}

void ehc_gnn_destroy(ehc_gnn *g) {
  if (!g) return;
  void *d[] = {g->p, g->m, g->v, g->grad, g->pb, g->in, g->u, g->y0, g->ybuf, g->G, g->du, g->mpart, g->epart,
               g->T, g->Tt, g->lpart, g->loss};
  for (void *q : d)
    if (q) cudaFree(q);
  if (g->host) cudaFreeHost(g->host);
  if (g->host_loss) cudaFreeHost(g->host_loss);
  delete g;
}

int ehc_gnn_set_params(ehc_gnn *g, ehc_ctx *hc, const float *params_host) {
  if (!g || !hc || !params_host) return EHC_E_INVAL;
  Ctx &c = hc->c;
  std::memcpy(g->host, params_host, sizeof(float) * kGnnParams);
  CK(cudaMemcpyAsync(g->p, g->host, sizeof(float) * kGnnParams, cudaMemcpyHostToDevice, c.stream));
  CK(cudaMemsetAsync(g->m, 0, sizeof(float) * kGnnParams, c.stream));
  CK(cudaMemsetAsync(g->v, 0, sizeof(float) * kGnnParams, c.stream));
  CK(gnn_params_to_bf16(c.stream, g->p, g->pb));
  CK(cudaStreamSynchronize(c.stream));
  g->t = 0;
  return EHC_OK;
}

int ehc_gnn_get_params(ehc_gnn *g, ehc_ctx *hc, float *params_host) {
  if (!g || !hc || !params_host) return EHC_E_INVAL;
  Ctx &c = hc->c;
  CK(cudaMemcpyAsync(g->host, g->p, sizeof(float) * kGnnParams, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  std::memcpy(params_host, g->host, sizeof(float) * kGnnParams);
  return EHC_OK;
}

int ehc_gnn_apply(ehc_gnn *g, ehc_ctx *hc, double kappa, const double *Y_dev, double *Yhat_dev, double *dY_dev) {
  if (!g || !hc || hc->c.n != g->n || (g->n > 0 && (!Y_dev || !Yhat_dev)) || !(kappa == kappa)) return EHC_E_INVAL;
  Ctx &c = hc->c;
  if (!c.built) return EHC_E_STATE;
  if (c.n == 0) return EHC_OK;
  CK(nn_gather(c, Y_dev, nullptr, g->T, nullptr, g->y0, false));
  CK(gnn_forward(c, g->pb, g->sigma, kappa, g->y0, g->in, g->u, g->T, g->ybuf, dY_dev ? g->Tt : nullptr));
  CK(launch_unpermute(c, g->T, Yhat_dev, 0));
  if (dY_dev) CK(launch_unpermute(c, g->Tt, dY_dev, 0));
  return EHC_OK;
}

int ehc_gnn_train_step(ehc_gnn *g, ehc_ctx *hc, double kappa, const double *Y_dev, const double *Tstar_dev,
                       float lr, float *loss_host, float *grad_host) {
  NvtxRange nvtx_range("ehc_gnn_train_step");
  if (!g || !hc || hc->c.n != g->n || g->n == 0 || !Y_dev || !Tstar_dev || !(kappa == kappa) || !(lr >= 0))
    return EHC_E_INVAL;
  Ctx &c = hc->c;
  if (!c.built) return EHC_E_STATE;
  CK(nn_gather(c, Y_dev, Tstar_dev, g->T, g->Tt, g->y0, false));
  CK(gnn_forward(c, g->pb, g->sigma, kappa, g->y0, g->in, g->u, g->T, g->ybuf, nullptr));
  CK(gnn_backward(c, g->pb, g->sigma, kappa, g->y0, g->in, g->u, g->T, g->Tt, g->G, g->du, g->lpart, g->loss,
                  g->mpart, g->epart, g->grad));
  if (grad_host) CK(cudaMemcpyAsync(g->host, g->grad, sizeof(float) * kGnnParams, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(g->host_loss, g->loss, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  if (lr > 0) {
    g->t += 1;
    CK(gnn_adam(c.stream, g->p, g->m, g->v, g->grad, lr, g->t, g->pb));
  }
  CK(cudaStreamSynchronize(c.stream));
  if (grad_host) std::memcpy(grad_host, g->host, sizeof(float) * kGnnParams);
  if (loss_host) *loss_host = (float)g->host_loss[0];
  return EHC_OK;
}

int ehc_batch_tuning(ehc_batch *b, int32_t *tile_threads, int32_t *grid_quarters) {
  if (!b || !tile_threads || !grid_quarters) return EHC_E_INVAL;
  *tile_threads = b->tile_nt;
  *grid_quarters = b->tile_nt ? b->tile_q : 0;
  return EHC_OK;
}

int ehc_tuning(ehc_ctx *h, int32_t *tile_threads, int32_t *grid_quarters) {
  if (!h || !tile_threads || !grid_quarters) return EHC_E_INVAL;
  *tile_threads = h->c.tile_nt;
  *grid_quarters = h->c.tile_nt ? h->c.tile_q : 0;
  return EHC_OK;
}

int ehc_cheb_set_corrector(ehc_cheb *w, ehc_gnn *g) {
  if (!w || (g && g->n != w->n)) return EHC_E_INVAL;
  w->corr = g;
  return EHC_OK;
}

}  // extern "C"
